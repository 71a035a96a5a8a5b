// Host-side launchers of the device kernels (one translation unit per kernel family).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "agile_internal.h"

namespace agile {

struct StageArgs;

// Per-stage update (macro-kernel), dispatched on physics / precision / limiter / flux.
cudaError_t launch_stage_hd(int real_bytes, int lim, int flux, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_mhd(int real_bytes, int lim, int flux, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_mhd_res(int real_bytes, int lim, int flux, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_srhd(int real_bytes, int lim, int flux, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_srhd_synge(int real_bytes, int lim, int flux, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_ffhd(int real_bytes, int lim, int flux, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_ffhd_htc(int real_bytes, int lim, int flux, const StageArgs& a, cudaStream_t s);

struct AuxArgs {
  int phys;                 // PhysKind (PH_SRHD_SYNGE for srhd with the Synge EOS)
  int real_bytes;
  double gamma;
  double cfl;
  double glm_alpha;
  const void* U;            // state pool
  void* Uw;                 // writable pool (kernels that update in place)
  const void* G;            // ghost slots of U
  void* Gw;
  void* FR;                 // flux registers
  const BlockDesc* bd;
  int nblk;
  int* status;
  const int* solve_of = nullptr;   // solve index per block (batched solves), nullptr = one solve
  int nsolve = 1;
  // work list of the per-block kernels (speeds, GLM decay, estimator): pool block of each of
  // the nblk work items, nullptr = blocks 0 .. nblk-1
  const int* wl = nullptr;
};

// Whether the stage kernel of a physics reads primitives from the recovery pass (SRHD).
inline bool phys_prim_pass(int phys) { return phys == PH_SRHD || phys == PH_SRHD_SYNGE; }
// Recovery pass before a stage launch: primitives and auxiliaries of a.U (the a.nblk work
// items of a.wl) into W and of the nslots ghost slots a.G into WG, with the same layouts;
// with speeds non-null also the CFL maxima of a.U per solve (a.solve_of), merged into
// speeds[solve][2] (the caller zeroes them).
cudaError_t launch_prim_pass(const AuxArgs& a, void* W, void* WG, int nslots, unsigned long long* speeds,
                             cudaStream_t s);
// Fill ghost slots of coarse-fine faces from U (restriction / limited prolongation).
cudaError_t launch_ghosts(const AuxArgs& a, const GhostTask* tasks, int ntasks, cudaStream_t s);
// Coarse-fine flux correction of the stage output a.Uw with stage weight b and dt.
cudaError_t launch_fixup(const AuxArgs& a, const FixupTask* tasks, int ntasks, double b,
                         const double* dtch, cudaStream_t s);
// Max signal-speed reduction of U into speeds[2] (double bits; caller zeroes them).
cudaError_t launch_speeds(const AuxArgs& a, unsigned long long* speeds, cudaStream_t s);
// dtch[solve] = {dt, c_h}: dt from the host value or (dt <= 0) cfl / max sum_d s_d / dx_d,
// for each of nsolve solves (speeds[solve][2]).
cudaError_t launch_set_dt(const unsigned long long* speeds, double* dtch, double dt_host,
                          double cfl, cudaStream_t s, int nsolve = 1, double rate_floor = 0.0);
// psi *= exp(-dt/2 c_h alpha / min dx) on every block.
cudaError_t launch_glm_decay(const AuxArgs& a, const double* dtch, cudaStream_t s);
// Loehner estimate: emax[nblk] (FP64, no FMA). With tols (per solve {refine threshold,
// coarsen threshold}, solve index a.solve_of[b] or 0) and margin >= 0 (a bound on the
// difference between the FP32 and the exact estimate of a cell), a block whose FP32 maximum
// is farther than margin from both of its thresholds gets that FP32 maximum (the same
// refinement decision), every other block the exact value.
cudaError_t launch_estimate(const AuxArgs& a, const int* vars, const double* weights, int nvars,
                            double eps, double* emax, cudaStream_t s, const double* tols = nullptr,
                            double margin = -1.0);
// The margin for launch_estimate's screen: four times the bound sum_i |w_i| (8 u / eps + 32 u),
// u = 2^-24, on the FP32 evaluation error of a cell's weighted estimate (-1: no screen).
inline double estimate_screen_margin(const double* weights, int nvars, double eps) {
  if (!(eps > 0.0)) return -1.0;
  double sw = 0.0;
  for (int i = 0; i < nvars; ++i) sw += weights[i] < 0.0 ? -weights[i] : weights[i];
  const double u = 1.0 / 16777216.0;
  return 4.0 * sw * (8.0 * u / eps + 32.0 * u);
}
// New pool from the old one (copy / prolong / restrict per block).
cudaError_t launch_regrid(const AuxArgs& old_pool, void* Unew, const RegridSrc* src, int nnew,
                          cudaStream_t s);
// Primitive (double) -> conserved (R) for the listed blocks; aux from primitives (SRHD).
cudaError_t launch_prim2cons(const AuxArgs& a, const double* prim, const int* blocks, int n,
                             cudaStream_t s);
// Conserved (double) -> pool (R) for all blocks; aux cleared.
cudaError_t launch_unpack(const AuxArgs& a, const double* cons, cudaStream_t s);
// Pool (R) -> conserved (double) [nblk][nv][4096], and aux [nblk][na][4096] if aux != nullptr.
cudaError_t launch_pack(const AuxArgs& a, double* cons, double* aux, cudaStream_t s);
// Per-block FP64 sums of every conserved variable times the cell volume: part[nblk][nv].
cudaError_t launch_sums(const AuxArgs& a, double* part, cudaStream_t s);
// Face-ghost view of one block: out[nt][20][20][20] (NaN at edges / corners).
cudaError_t launch_halo(const AuxArgs& a, int block, double* out, cudaStream_t s);

// Radiative-loss table (Townsend exact integration, see cooling.cu): per segment
// [ln T_k, T_k / L_k, e = 1 - alpha_k, W_k = int_{T_k}^{T_{k+1}} dT / Lambda, T_{k+1},
//  L_{k+1} / T_{k+1}, L_k / T_k, ln T_{k+1}].
constexpr int COOL_SEG = 8;
constexpr int COOL_MAX_NODES = 4096;
struct CoolDev {
  int nseg = 0;        // segments (nodes - 1); 0 = no losses
  int uniform = 0;     // nodes uniform in ln T
  double lnT0 = 0.0, idln = 0.0, T0 = 0.0;
  double g1 = 0.0;     // gamma - 1: a step consumes (gamma - 1) rho dt of int dT / Lambda
  // the same four rounded to FP32 on the host: the FP32 kernel reads these, so that it never
  // converts FP64 values per cell (conversions run on the FP64 units)
  float lnT0f = 0.0f, idlnf = 0.0f, T0f = 0.0f, g1f = 0.0f;
};
struct CoolHost : CoolDev {
  std::vector<double> segd;
  std::vector<float> segf;
};
// Validates the table (2..COOL_MAX_NODES nodes, T increasing, T and Lambda positive and
// finite, every derived segment quantity finite in the stencil precision real_bytes) and
// fills out; returns nonzero when it is invalid.
int build_cool_table(const double* T, const double* L, int n, double gamma, int real_bytes, CoolHost* out);
// Losses over frac * dt (dt per solve from dtch) on the hd / mhd pool a.Uw; with speeds
// != nullptr also the CFL speed maxima of the result (caller zeroes them).
cudaError_t launch_cooling(const AuxArgs& a, const CoolDev& c, const void* seg, const double* dtch,
                           double frac, unsigned long long* speeds, cudaStream_t s);

int phys_nvar(int phys);
int phys_naux(int phys);

}  // namespace agile
