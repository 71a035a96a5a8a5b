// C ABI of the block-AMR library: mesh lifecycle, device pools, the SSPRK step driver
// (paper Fig. 2), regrid (Figs. 1-2), state transfer and diagnostics.
#include <cuda.h>
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/agile.h"
#include "kernels.cuh"
#include "launch.h"
#include "mesh.h"

using namespace agile;

// Deterministic compensated total of per-block sums (defined with the conserved-sum calls).
__global__ void sums_total_kernel(const double* part, int nblk, int nv, double* totals);

struct agile_mesh {
  agile_config cfg;
  cudaStream_t stream = nullptr;
  agile_allocator alloc{};
  bool default_alloc = true;
  int nv = 5, na = 0, nt = 5, rb = 8;
  HostMesh* mesh = nullptr;
  int nblk = 0;
  void* U[3] = {nullptr, nullptr, nullptr};
  void* G = nullptr;
  void* FR = nullptr;
  int nslots = 0;
  BlockDesc* d_bd = nullptr;
  int* d_wl = nullptr;             // stage kernel work order (blocks by level, z-slab, 2-D Morton)
  GhostTask* d_ghosts = nullptr;
  FixupTask* d_fix = nullptr;
  int nghost = 0, nfix = 0;
  int* d_status = nullptr;
  unsigned long long* d_speeds = nullptr;
  double* d_dtch = nullptr;
  int* d_work = nullptr;            // per-stage block counters of the persistent launches
  int* d_vars = nullptr;
  double* d_weights = nullptr;
  bool speeds_valid = false;
  agile_ic_fn ic = nullptr;
  void* ic_user = nullptr;
  std::string err;
  CUtensorMap tmap[3];
  // SRHD: primitives of the stage input from the recovery pass (pool and ghost slots) and
  // the tensor map the stage kernel's TMA reads them through
  void* W = nullptr;
  void* WG = nullptr;
  CUtensorMap tmapW;
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_cat;          // phase of each event pair (PHASE_*)
  long long stage_launches = 0, total_launches = 0;
  long long phase_launches[4] = {0, 0, 0, 0};
  CoolHost cool;                    // radiative-loss table (nseg == 0: no losses)
  void* d_cool = nullptr;           // its segments in the stencil precision
  double* d_sums = nullptr;         // per-block sums and totals of agile_conserved_sums (kept)
  size_t d_sums_cap = 0;            // its capacity in doubles
};

namespace {

// Device address of a page-locked host buffer (cudaHostAlloc, cudaHostRegister): under
// unified addressing kernels read and write it directly, so a transfer needs no staging copy
// in device memory. nullptr for pageable memory (the caller stages through a copy).
static void* pinned_view(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();              // clear the query's error: the caller stages the copy
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

void* dalloc(agile_mesh* m, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (m->default_alloc) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, m->stream) != cudaSuccess) return nullptr;
    return p;
  }
  return m->alloc.alloc(bytes, (void*)m->stream, m->alloc.ctx);
}

void dfree(agile_mesh* m, void*& p) {
  if (!p) return;
  if (m->default_alloc) cudaFreeAsync(p, m->stream);
  else m->alloc.free(p, (void*)m->stream, m->alloc.ctx);
  p = nullptr;
}

template <typename T>
void dfree_t(agile_mesh* m, T*& p) {
  void* q = (void*)p;
  dfree(m, q);
  p = nullptr;
}

agile_status fail(agile_mesh* m, agile_status s, const std::string& msg) {
  if (m) m->err = msg;
  return s;
}

// Phases timed with CUDA events when kernel timing is on: the stage (update) kernel, the
// coarse-fine ghost fill, the flux fix-up and the refinement estimator.
enum : int { PHASE_STAGE = 0, PHASE_GHOST = 1, PHASE_FIXUP = 2, PHASE_ESTIMATE = 3 };

cudaEvent_t phase_begin(agile_mesh* m) {
  if (!m->timing) return nullptr;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  cudaEventRecord(e, m->stream);
  return e;
}

void phase_end(agile_mesh* m, cudaEvent_t e0, int phase) {
  if (!e0) return;
  cudaEvent_t e1 = nullptr;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return;
  }
  cudaEventRecord(e1, m->stream);
  m->ev.push_back(e0);
  m->ev.push_back(e1);
  m->ev_cat.push_back(phase);
  m->phase_launches[phase]++;
}

#define CK(m, call)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail((m), AGILE_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_));        \
  } while (0)

size_t pool_bytes(const agile_mesh* m, int nblk) {
  return (size_t)nblk * m->nt * NCELL * m->rb;
}

// Internal physics kind: the srhd module with the Synge EOS has its own device trait.
int phys_kind(const agile_config& c) {
  if (c.physics == AGILE_FFHD) return PH_FFHD;
  if (c.physics == AGILE_FFHD_HTC) return PH_FFHD_HTC;
  return c.physics == AGILE_SRHD && c.eos == AGILE_EOS_SYNGE ? PH_SRHD_SYNGE : c.physics;
}

int cfg_nvar(const agile_config& c) {
  return c.physics == AGILE_MHD_GLM ? 9 : (c.physics == AGILE_FFHD ? 6 : (c.physics == AGILE_FFHD_HTC ? 7 : 5));
}

// Scheme restrictions shared by meshes and batches: the solvers per module of paper
// Table 1 (TVDLF for srhd and ffhd, HLLC for hd), the Synge EOS for srhd only, ffhd on
// uniform meshes, a finite non-negative conduction coefficient.
bool scheme_ok(const agile_config& c) {
  const bool ffhd = c.physics == AGILE_FFHD || c.physics == AGILE_FFHD_HTC;
  if (c.physics < 0 || c.physics > 4 || (c.limiter != 0 && c.limiter != 1) || c.flux < 0 || c.flux > 2 ||
      (c.rk != 2 && c.rk != 3) || (c.real_bytes != 4 && c.real_bytes != 8) || !(c.gamma > 1.0) ||
      !(c.cfl > 0.0))
    return false;
  if ((c.physics == AGILE_SRHD || ffhd) && c.flux != AGILE_TVDLF) return false;
  if (c.flux == AGILE_HLLC && c.physics != AGILE_HD) return false;
  if (c.eos != AGILE_EOS_IDEAL && !(c.eos == AGILE_EOS_SYNGE && c.physics == AGILE_SRHD)) return false;
  if (ffhd && c.max_level != 1) return false;
  if (c.physics == AGILE_FFHD_HTC && !(c.htc_kappa0 >= 0.0 && c.htc_kappa0 < 1e300)) return false;
  if (!(c.eta >= 0.0 && c.eta < 1e300) || (c.eta > 0.0 && c.physics != AGILE_MHD_GLM)) return false;
  return true;
}

// 2 eta sum_d dx_d^-2 at the finest level of the mesh (0 without resistivity): the largest
// rate of the resistive diffusion term, which bounds the step like the signal speeds do.
double resistive_rate(const agile_config& c, int finest_level) {
  if (!(c.eta > 0.0)) return 0.0;
  double r = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double dx = (c.xmax[d] - c.xmin[d]) / ((double)c.base_blocks[d] * NB * (double)(1 << (finest_level - 1)));
    r += 1.0 / (dx * dx);
  }
  return 2.0 * c.eta * r;
}

AuxArgs aux_args(agile_mesh* m, void* U) {
  AuxArgs a;
  a.phys = phys_kind(m->cfg);
  a.real_bytes = m->rb;
  a.gamma = m->cfg.gamma;
  a.cfl = m->cfg.cfl;
  a.glm_alpha = m->cfg.glm_alpha;
  a.U = U;
  a.Uw = U;
  a.G = m->G;
  a.Gw = m->G;
  a.FR = m->FR;
  a.bd = m->d_bd;
  a.nblk = m->nblk;
  a.status = m->d_status;
  return a;
}

agile_status check_status(agile_mesh* m) {
  CK(m, cudaStreamSynchronize(m->stream));
  int st = 0;
  CK(m, cudaMemcpy(&st, m->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    CK(m, cudaMemset(m->d_status, 0, sizeof(int)));
    if (st & ST_ETIMEOUT) return fail(m, AGILE_ETIMEOUT, "a bounded wait for a TMA plane gave up");
    if (st & ST_ENOCONV) return fail(m, AGILE_ENOCONV, "primitive recovery did not converge");
    return fail(m, AGILE_EUNPHYS, "non-positive density or pressure on the device");
  }
  return AGILE_OK;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// Tensor map of one state pool as a 4-D array (x, y, z, block * var) whose TMA box is one
// z-plane of every variable of a block: {16, 16, 1, nvar + naux}.
agile_status make_tmap(agile_mesh* m, void* U, CUtensorMap* out) {
  memset(out, 0, sizeof(*out));
  if (!U) return AGILE_OK;
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(m, AGILE_ECUDA, "cuTensorMapEncodeTiled unavailable");
  const cuuint64_t dims[4] = {16, 16, 16, (cuuint64_t)m->nblk * m->nt};
  const cuuint64_t strides[3] = {(cuuint64_t)m->rb * 16, (cuuint64_t)m->rb * 256, (cuuint64_t)m->rb * 4096};
  const cuuint32_t box[4] = {16, 16, 1, (cuuint32_t)m->nt};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(out, m->rb == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, U,
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(m, AGILE_ECUDA, "cuTensorMapEncodeTiled failed");
  return AGILE_OK;
}

// (Re)build descriptors, slots and scratch for the current host mesh; U[0] must already
// hold nblk blocks.
// 2-D Morton code of (x, y) (16 bits each).
uint64_t morton2(uint32_t x, uint32_t y) {
  uint64_t c = 0;
  for (int i = 0; i < 16; ++i) c |= (uint64_t)((x >> i) & 1) << (2 * i) | (uint64_t)((y >> i) & 1) << (2 * i + 1);
  return c;
}

// Order in which the stage kernel's persistent CTAs take the blocks: by level, then by z
// index, then in 2-D Morton order within the z-slab. A slab's blocks run together, so the
// x/y halos a block reads belong to blocks that run at the same time and the z halos to the
// slabs just before and after it, which keeps the halo re-reads in L2 (the pool itself stays
// in 3-D Morton order).
std::vector<int> slab_order(const HostMesh& hm) {
  const auto& keys = hm.blocks();
  std::vector<int> w(keys.size());
  for (size_t i = 0; i < keys.size(); ++i) w[i] = (int)i;
  std::stable_sort(w.begin(), w.end(), [&](int a, int b) {
    const Key& p = keys[a];
    const Key& q = keys[b];
    if (p.lev != q.lev) return p.lev < q.lev;
    if (p.z != q.z) return p.z < q.z;
    return morton2(p.x, p.y) < morton2(q.x, q.y);
  });
  return w;
}

agile_status rebuild(agile_mesh* m) {
  std::vector<BlockDesc> desc;
  std::vector<GhostTask> ghosts;
  std::vector<FixupTask> fix;
  std::string err;
  int nslots = 0;
  m->mesh->build_descs(&desc, &ghosts, &fix, &nslots, &err);
  if (!err.empty()) return fail(m, AGILE_EINVAL, err);
  m->nblk = (int)desc.size();
  dfree_t(m, m->d_bd);
  dfree_t(m, m->d_ghosts);
  dfree_t(m, m->d_fix);
  dfree(m, m->G);
  dfree(m, m->FR);
  dfree(m, m->U[1]);
  dfree(m, m->U[2]);
  dfree(m, m->W);
  dfree(m, m->WG);
  dfree_t(m, m->d_wl);
  const std::vector<int> order = slab_order(*m->mesh);
  const bool prim_pass = phys_prim_pass(phys_kind(m->cfg));
  if (prim_pass) {
    m->W = dalloc(m, pool_bytes(m, m->nblk));
    m->WG = dalloc(m, (size_t)std::max(nslots, 1) * m->nt * 512 * m->rb);
    if (!m->W || !m->WG) return fail(m, AGILE_ENOMEM, "device allocation failed");
  }
  m->d_wl = (int*)dalloc(m, order.size() * sizeof(int));
  m->d_bd = (BlockDesc*)dalloc(m, desc.size() * sizeof(BlockDesc));
  m->d_ghosts = (GhostTask*)dalloc(m, ghosts.size() * sizeof(GhostTask));
  m->d_fix = (FixupTask*)dalloc(m, fix.size() * sizeof(FixupTask));
  m->G = dalloc(m, (size_t)nslots * m->nt * 512 * m->rb);
  m->FR = dalloc(m, (size_t)nslots * m->nv * 256 * m->rb);
  m->U[1] = dalloc(m, pool_bytes(m, m->nblk));
  m->U[2] = m->cfg.rk == 3 ? dalloc(m, pool_bytes(m, m->nblk)) : nullptr;
  if (!m->d_bd || !m->d_wl || !m->d_ghosts || !m->d_fix || !m->G || !m->FR || !m->U[1] ||
      (m->cfg.rk == 3 && !m->U[2]))
    return fail(m, AGILE_ENOMEM, "device allocation failed");
  CK(m, cudaMemcpyAsync(m->d_bd, desc.data(), desc.size() * sizeof(BlockDesc), cudaMemcpyHostToDevice, m->stream));
  if (!order.empty())
    CK(m, cudaMemcpyAsync(m->d_wl, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, m->stream));
  if (!ghosts.empty())
    CK(m, cudaMemcpyAsync(m->d_ghosts, ghosts.data(), ghosts.size() * sizeof(GhostTask), cudaMemcpyHostToDevice, m->stream));
  if (!fix.empty())
    CK(m, cudaMemcpyAsync(m->d_fix, fix.data(), fix.size() * sizeof(FixupTask), cudaMemcpyHostToDevice, m->stream));
  m->nghost = (int)ghosts.size();
  m->nfix = (int)fix.size();
  m->nslots = nslots;
  CK(m, cudaStreamSynchronize(m->stream));   // host vectors go out of scope
  m->speeds_valid = false;
  for (int i = 0; i < 3; ++i) {
    agile_status s = make_tmap(m, m->U[i], &m->tmap[i]);
    if (s) return s;
  }
  agile_status sw = make_tmap(m, m->W, &m->tmapW);
  if (sw) return sw;
  return AGILE_OK;
}

agile_status fill_ghosts(agile_mesh* m, void* U) {
  if (m->nghost == 0) return AGILE_OK;
  AuxArgs a = aux_args(m, U);
  cudaEvent_t e0 = phase_begin(m);
  CK(m, launch_ghosts(a, m->d_ghosts, m->nghost, m->stream));
  phase_end(m, e0, PHASE_GHOST);
  m->total_launches++;
  return AGILE_OK;
}

// Evaluate the initial condition on the listed blocks (host callback, then prim -> cons on
// the device), in chunks to bound host and device staging.
// Initial state of the listed blocks: primitives from the mesh's callback at the cell centres,
// or (prim_src non-null) from the host array prim_src[i][nv][16^3] for the i-th listed
// block; converted to conserved variables on the device.
agile_status apply_ic(agile_mesh* m, void* U, const std::vector<int>& blocks, const double* prim_src = nullptr) {
  const int chunk = 256;
  std::vector<double> prim(prim_src ? 0 : (size_t)chunk * m->nv * NCELL);   // callback staging
  const void* prim_view = prim_src ? pinned_view(prim_src) : nullptr;
  std::vector<double> xs(NCELL), ys(NCELL), zs(NCELL);
  double* d_prim = (double*)dalloc(m, (size_t)chunk * m->nv * NCELL * sizeof(double));
  int* d_blocks = (int*)dalloc(m, chunk * sizeof(int));
  if (!d_prim || !d_blocks) return fail(m, AGILE_ENOMEM, "device allocation failed");
  const auto& keys = m->mesh->blocks();
  for (size_t c0 = 0; c0 < blocks.size(); c0 += chunk) {
    const int n = (int)std::min(blocks.size() - c0, (size_t)chunk);
    for (int i = 0; i < n && !prim_src; ++i) {
      const Key& k = keys[blocks[c0 + i]];
      const double dx = m->mesh->dx(k.lev, 0), dy = m->mesh->dx(k.lev, 1), dz = m->mesh->dx(k.lev, 2);
      for (int z = 0; z < NB; ++z)
        for (int y = 0; y < NB; ++y)
          for (int x = 0; x < NB; ++x) {
            const int c = z * 256 + y * 16 + x;
            xs[c] = m->cfg.xmin[0] + ((double)(k.x * NB + x) + 0.5) * dx;
            ys[c] = m->cfg.xmin[1] + ((double)(k.y * NB + y) + 0.5) * dy;
            zs[c] = m->cfg.xmin[2] + ((double)(k.z * NB + z) + 0.5) * dz;
          }
      m->ic(xs.data(), ys.data(), zs.data(), NCELL, prim.data() + (size_t)i * m->nv * NCELL, m->ic_user);
    }
    const double* src = prim_src ? prim_src + c0 * m->nv * NCELL : prim.data();
    // page-locked primitives are read in place by the conversion, others staged first
    const double* dsrc = prim_view ? (const double*)prim_view + c0 * m->nv * NCELL : d_prim;
    if (!prim_view)
      CK(m, cudaMemcpyAsync(d_prim, src, (size_t)n * m->nv * NCELL * sizeof(double), cudaMemcpyHostToDevice,
                            m->stream));
    CK(m, cudaMemcpyAsync(d_blocks, blocks.data() + c0, n * sizeof(int), cudaMemcpyHostToDevice, m->stream));
    AuxArgs a = aux_args(m, U);
    CK(m, launch_prim2cons(a, dsrc, d_blocks, n, m->stream));
    m->total_launches++;
    // the next chunk reuses the device staging in stream order; the callback path also
    // waits because its host buffer is refilled for the next chunk
    if (!prim_src) CK(m, cudaStreamSynchronize(m->stream));
  }
  dfree_t(m, d_prim);
  dfree_t(m, d_blocks);
  return AGILE_OK;
}

// Resistive rate of the mesh at its current finest level (leaves are sorted by level).
double mesh_res_rate(const agile_mesh* m) {
  if (!(m->cfg.eta > 0.0) || m->mesh->blocks().empty()) return 0.0;
  return resistive_rate(m->cfg, m->mesh->blocks().back().lev);
}

agile_status ensure_speeds(agile_mesh* m) {
  if (m->speeds_valid) return AGILE_OK;
  CK(m, cudaMemsetAsync(m->d_speeds, 0, 2 * sizeof(unsigned long long), m->stream));
  AuxArgs a = aux_args(m, m->U[0]);
  CK(m, launch_speeds(a, m->d_speeds, m->stream));
  m->total_launches++;
  m->speeds_valid = true;
  return AGILE_OK;
}

agile_status do_regrid(agile_mesh* m, const std::vector<int>& flags, int init, int* nr, int* nc) {
  RegridPlan plan = m->mesh->plan(flags);
  if (nr) *nr = plan.n_refined;
  if (nc) *nc = plan.n_coarsened;
  if (plan.n_refined == 0 && plan.n_coarsened == 0) return AGILE_OK;
  agile_status s = fill_ghosts(m, m->U[0]);
  if (s) return s;
  const int nnew = (int)plan.blocks.size();
  void* Unew = dalloc(m, pool_bytes(m, nnew));
  RegridSrc* d_src = (RegridSrc*)dalloc(m, plan.src.size() * sizeof(RegridSrc));
  if (!Unew || !d_src) return fail(m, AGILE_ENOMEM, "device allocation failed");
  CK(m, cudaMemcpyAsync(d_src, plan.src.data(), plan.src.size() * sizeof(RegridSrc), cudaMemcpyHostToDevice, m->stream));
  AuxArgs a = aux_args(m, m->U[0]);
  CK(m, launch_regrid(a, Unew, d_src, nnew, m->stream));
  m->total_launches++;
  CK(m, cudaStreamSynchronize(m->stream));
  dfree_t(m, d_src);
  dfree(m, m->U[0]);
  m->U[0] = Unew;
  m->mesh->apply(plan);
  s = rebuild(m);
  if (s) return s;
  if (init && m->ic) {
    s = apply_ic(m, m->U[0], plan.created);
    if (s) return s;
  }
  return check_status(m);
}

}  // namespace

namespace {
// Bounded-wait check: one thread initialises an mbarrier that expects one arrival, nobody
// arrives, and the thread polls it at most `limit` times (the same bounded wait the stage
// kernel uses for its TMA planes), then records whether the wait ran out.
__global__ void selftest_wait_kernel(uint32_t limit, int* out) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    out[0] = mbar_wait(&bar, 0, limit) ? 0 : 1;
  }
}

// Accuracy of the FP64 stencil quotient rdiv(a, s) against the IEEE quotient: per element the
// distance in units of the last place of the IEEE result (measured towards rdiv's result),
// maxima over all elements as non-negative doubles through their ordered bit patterns.
__global__ void selftest_rcp64_kernel(const double* __restrict__ s, const double* __restrict__ a, size_t n,
                                      unsigned long long* out) {
  double mu = 0.0, mr = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double q0 = __ddiv_rn(a[i], s[i]);
    const double q1 = rdiv(a[i], s[i]);
    if (q1 != q0) {
      const double step = fabs(nextafter(q0, q1) - q0);
      mu = fmax(mu, fabs(q1 - q0) / step);
      mr = fmax(mr, fabs(q1 - q0) / fabs(q0));
    }
  }
  atomicMax(out, (unsigned long long)__double_as_longlong(mu));
  atomicMax(out + 1, (unsigned long long)__double_as_longlong(mr));
}
}  // namespace

extern "C" {

agile_status agile_selftest_rcp64(const double* s, const double* a, size_t n, void* stream, double* max_ulps,
                                  double* max_rel) {
  if (!s || !a || !max_ulps || !max_rel || n == 0 || n > ((size_t)1 << 26)) return AGILE_EINVAL;
  for (size_t i = 0; i < n; ++i) {
    const double v = std::fabs(s[i]);
    if (!(v >= DBL_MIN && v < std::ldexp(1.0, 1022)) || !std::isfinite(a[i])) return AGILE_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double *ds = nullptr, *da = nullptr;
  unsigned long long* dout = nullptr;
  cudaError_t e = cudaMallocAsync(&ds, n * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&da, n * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&dout, 2 * sizeof(unsigned long long), st);
  unsigned long long h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(ds, s, n * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(da, a, n * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dout, 0, 2 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, 4096);
    selftest_rcp64_kernel<<<grid, 256, 0, st>>>(ds, da, n, dout);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, dout, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (ds) cudaFreeAsync(ds, st);
  if (da) cudaFreeAsync(da, st);
  if (dout) cudaFreeAsync(dout, st);
  if (e != cudaSuccess) return AGILE_ECUDA;
  std::memcpy(max_ulps, &h[0], sizeof(double));
  std::memcpy(max_rel, &h[1], sizeof(double));
  return AGILE_OK;
}

const char* agile_version(void) { return "agile-gb300 1.0 (sm_103a)"; }

const char* agile_last_error(const agile_mesh* m) { return m ? m->err.c_str() : "null mesh"; }

agile_status agile_selftest_bounded_wait(void* stream, unsigned int limit, int* timed_out) {
  if (!timed_out || limit == 0 || limit > (1u << 24)) return AGILE_EINVAL;
  int* d = nullptr;
  if (cudaMallocAsync(&d, sizeof(int), (cudaStream_t)stream) != cudaSuccess) return AGILE_ENOMEM;
  selftest_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(limit, d);
  int h = -1;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  cudaFreeAsync(d, (cudaStream_t)stream);
  if (e != cudaSuccess) return AGILE_ECUDA;
  *timed_out = h;
  return h ? AGILE_ETIMEOUT : AGILE_OK;
}

agile_status agile_mesh_create(const agile_config* cfg, const agile_allocator* alloc, void* stream,
                               agile_mesh** out) {
  if (!cfg || !out) return AGILE_EINVAL;
  *out = nullptr;
  if (!scheme_ok(*cfg) || cfg->max_level < 1 || cfg->max_level > 12 || cfg->refine_nvars < 0 ||
      cfg->refine_nvars > 9)
    return AGILE_EINVAL;
  for (int d = 0; d < 3; ++d) {
    if (cfg->base_blocks[d] < 1 || cfg->base_blocks[d] > 4096 || !(cfg->xmax[d] > cfg->xmin[d]))
      return AGILE_EINVAL;
    const bool p0 = cfg->bc[2 * d] == AGILE_PERIODIC, p1 = cfg->bc[2 * d + 1] == AGILE_PERIODIC;
    if (p0 != p1) return AGILE_EINVAL;
    for (int s = 0; s < 2; ++s)
      if (cfg->bc[2 * d + s] < 0 || cfg->bc[2 * d + s] > 2) return AGILE_EINVAL;
  }
  const int nvar = cfg_nvar(*cfg);
  for (int i = 0; i < cfg->refine_nvars; ++i)
    if (cfg->refine_vars[i] < 0 || cfg->refine_vars[i] >= nvar) return AGILE_EINVAL;
  agile_mesh* m = new agile_mesh();
  m->cfg = *cfg;
  m->stream = (cudaStream_t)stream;
  if (alloc && alloc->alloc && alloc->free) {
    m->alloc = *alloc;
    m->default_alloc = false;
  }
  m->nv = nvar;
  m->na = cfg->physics == AGILE_SRHD ? 2 : 0;
  m->nt = m->nv + m->na;
  m->rb = cfg->real_bytes;
  m->mesh = new HostMesh(cfg->base_blocks, cfg->max_level, cfg->bc, cfg->xmin, cfg->xmax);
  m->nblk = (int)m->mesh->blocks().size();
  m->U[0] = dalloc(m, pool_bytes(m, m->nblk));
  m->d_status = (int*)dalloc(m, sizeof(int));
  m->d_speeds = (unsigned long long*)dalloc(m, 2 * sizeof(unsigned long long));
  m->d_dtch = (double*)dalloc(m, 2 * sizeof(double));
  m->d_work = (int*)dalloc(m, 4 * sizeof(int));
  m->d_vars = (int*)dalloc(m, 9 * sizeof(int));
  m->d_weights = (double*)dalloc(m, 9 * sizeof(double));
  if (!m->U[0] || !m->d_status || !m->d_speeds || !m->d_dtch || !m->d_work || !m->d_vars || !m->d_weights) {
    agile_mesh_destroy(m);
    return AGILE_ENOMEM;
  }
  if (cudaMemsetAsync(m->d_status, 0, sizeof(int), m->stream) != cudaSuccess ||
      cudaMemsetAsync(m->U[0], 0, pool_bytes(m, m->nblk), m->stream) != cudaSuccess ||
      cudaMemcpyAsync(m->d_vars, cfg->refine_vars, 9 * sizeof(int), cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
      cudaMemcpyAsync(m->d_weights, cfg->refine_weights, 9 * sizeof(double), cudaMemcpyHostToDevice, m->stream) != cudaSuccess) {
    agile_mesh_destroy(m);
    return AGILE_ECUDA;
  }
  if (rebuild(m) != AGILE_OK) {
    agile_mesh_destroy(m);
    return AGILE_ECUDA;
  }
  *out = m;
  return AGILE_OK;
}

void agile_mesh_destroy(agile_mesh* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  for (int i = 0; i < 3; ++i) dfree(m, m->U[i]);
  dfree(m, m->G);
  dfree(m, m->FR);
  dfree_t(m, m->d_bd);
  dfree_t(m, m->d_wl);
  dfree(m, m->W);
  dfree(m, m->WG);
  dfree_t(m, m->d_ghosts);
  dfree_t(m, m->d_fix);
  dfree_t(m, m->d_status);
  dfree_t(m, m->d_speeds);
  dfree_t(m, m->d_dtch);
  dfree_t(m, m->d_work);
  dfree_t(m, m->d_sums);
  dfree_t(m, m->d_vars);
  dfree_t(m, m->d_weights);
  dfree(m, m->d_cool);
  for (cudaEvent_t e : m->ev) cudaEventDestroy(e);
  cudaStreamSynchronize(m->stream);
  delete m->mesh;
  delete m;
}

agile_status agile_set_state(agile_mesh* m, agile_ic_fn ic, void* user) {
  if (!m || !ic) return fail(m, AGILE_EINVAL, "null argument");
  m->ic = ic;
  m->ic_user = user;
  std::vector<int> all(m->nblk);
  for (int i = 0; i < m->nblk; ++i) all[i] = i;
  agile_status s = apply_ic(m, m->U[0], all);
  if (s) return s;
  m->speeds_valid = false;
  return check_status(m);
}

agile_status agile_set_state_blocks(agile_mesh* m, const double* cons, size_t nblk) {
  if (!m || !cons) return fail(m, AGILE_EINVAL, "null argument");
  if ((int)nblk != m->nblk) return fail(m, AGILE_EINVAL, "block count does not match the mesh");
  if (const void* dv = pinned_view(cons)) {   // page-locked: the unpack reads it in place
    AuxArgs a = aux_args(m, m->U[0]);
    CK(m, launch_unpack(a, (const double*)dv, m->stream));
    m->total_launches++;
    CK(m, cudaStreamSynchronize(m->stream));
    m->speeds_valid = false;
    return AGILE_OK;
  }
  const size_t bytes = nblk * m->nv * NCELL * sizeof(double);
  double* d = (double*)dalloc(m, bytes);
  if (!d) return fail(m, AGILE_ENOMEM, "device allocation failed");
  CK(m, cudaMemcpyAsync(d, cons, bytes, cudaMemcpyHostToDevice, m->stream));
  AuxArgs a = aux_args(m, m->U[0]);
  CK(m, launch_unpack(a, d, m->stream));
  m->total_launches++;
  CK(m, cudaStreamSynchronize(m->stream));
  dfree_t(m, d);
  m->speeds_valid = false;
  return AGILE_OK;
}

agile_status agile_set_state_prims(agile_mesh* m, const double* prim, size_t nblk) {
  if (!m || !prim) return fail(m, AGILE_EINVAL, "null argument");
  if ((int)nblk != m->nblk) return fail(m, AGILE_EINVAL, "block count does not match the mesh");
  std::vector<int> all(nblk);
  for (size_t i = 0; i < nblk; ++i) all[i] = (int)i;
  m->ic = nullptr;      // no callback for later regrid(init=1) re-evaluation
  m->ic_user = nullptr;
  agile_status s = apply_ic(m, m->U[0], all, prim);
  if (s) return s;
  m->speeds_valid = false;
  return check_status(m);
}

agile_status agile_cfl_dt(agile_mesh* m, double* dt_out) {
  if (!m || !dt_out) return fail(m, AGILE_EINVAL, "null argument");
  agile_status s = ensure_speeds(m);
  if (s) return s;
  unsigned long long h[2];
  CK(m, cudaMemcpyAsync(h, m->d_speeds, sizeof(h), cudaMemcpyDeviceToHost, m->stream));
  s = check_status(m);
  if (s) return s;
  double smax;
  memcpy(&smax, &h[0], sizeof(double));
  if (!(smax > 0.0)) return fail(m, AGILE_EUNPHYS, "zero or invalid signal speed");
  *dt_out = m->cfg.cfl / std::max(smax, mesh_res_rate(m));
  return AGILE_OK;
}

agile_status agile_max_speeds(agile_mesh* m, double* sum_over_dx, double* cmax) {
  if (!m) return AGILE_EINVAL;
  agile_status s = ensure_speeds(m);
  if (s) return s;
  unsigned long long h[2];
  CK(m, cudaMemcpyAsync(h, m->d_speeds, sizeof(h), cudaMemcpyDeviceToHost, m->stream));
  s = check_status(m);
  if (s) return s;
  if (sum_over_dx) memcpy(sum_over_dx, &h[0], sizeof(double));
  if (cmax) memcpy(cmax, &h[1], sizeof(double));
  return AGILE_OK;
}

agile_status agile_step(agile_mesh* m, double dt) {
  if (!m) return AGILE_EINVAL;
  // SRHD (a recovery pass before each stage): the first stage's pass also reduces the CFL
  // maxima of U^n and dt is set after it, instead of a reduction at the end of the step
  const bool lead = m->W != nullptr;
  agile_status s = AGILE_OK;
  if (!lead) {
    s = ensure_speeds(m);
    if (s) return s;
    CK(m, launch_set_dt(m->d_speeds, m->d_dtch, dt, m->cfg.cfl, m->stream, 1, mesh_res_rate(m)));
    m->total_launches++;
  }
  CK(m, cudaMemsetAsync(m->d_work, 0, 4 * sizeof(int), m->stream));
  const bool mhd = m->cfg.physics == AGILE_MHD_GLM;
  if (mhd) {
    AuxArgs a = aux_args(m, m->U[0]);
    CK(m, launch_glm_decay(a, m->d_dtch, m->stream));
    m->total_launches++;
  }
  static const double w2[2][2] = {{0.0, 1.0}, {0.5, 0.5}};
  static const double w3[3][2] = {{0.0, 1.0}, {0.75, 0.25}, {1.0 / 3.0, 2.0 / 3.0}};
  const int nst = m->cfg.rk;
  const bool fuse = m->nfix == 0;
  const bool cool = m->cool.nseg > 0;
  const bool speeds_in_stage = fuse && !cool && !lead;   // else the post-step pass reduces them
  if (cool) {                                   // first Strang half of the losses
    AuxArgs a = aux_args(m, m->U[0]);
    CK(m, launch_cooling(a, m->cool, m->d_cool, m->d_dtch, 0.5, nullptr, m->stream));
    m->total_launches++;
  }
  for (int st = 0; st < nst; ++st) {
    const bool last = st == nst - 1;
    void* Us = st == 0 ? m->U[0] : m->U[st];
    void* Uo = last ? m->U[0] : m->U[st + 1];
    s = fill_ghosts(m, Us);
    if (s) return s;
    if (last && speeds_in_stage) CK(m, cudaMemsetAsync(m->d_speeds, 0, 2 * sizeof(unsigned long long), m->stream));
    StageArgs A;
    A.Us = Us;
    A.Un = m->U[0];
    A.Uout = Uo;
    A.bd = m->d_bd;
    A.gs = m->G;
    A.fr = m->nfix ? m->FR : nullptr;
    A.dtch = m->d_dtch;
    A.a = nst == 2 ? w2[st][0] : w3[st][0];
    A.b = nst == 2 ? w2[st][1] : w3[st][1];
    A.gamma = m->cfg.gamma;
    A.glm_alpha = m->cfg.glm_alpha;
    A.htc_kappa0 = m->cfg.htc_kappa0;
    A.eta = m->cfg.eta;
    A.glm_post = (mhd && last && fuse) ? 1 : 0;
    A.nblk = m->nblk;
    A.wl = m->d_wl;
    A.status = m->d_status;
    A.speeds = (last && speeds_in_stage) ? m->d_speeds : nullptr;
    A.tmap = &m->tmap[st == 0 ? 0 : st];
    A.solve_of = nullptr;
    A.work = m->d_work + st;
    cudaEvent_t e0 = phase_begin(m);
    if (m->W) {                      // one recovery per stored cell, read by the stage kernel
      AuxArgs pa = aux_args(m, Us);
      if (st == 0) CK(m, cudaMemsetAsync(m->d_speeds, 0, 2 * sizeof(unsigned long long), m->stream));
      CK(m, launch_prim_pass(pa, m->W, m->WG, m->nslots, st == 0 ? m->d_speeds : nullptr, m->stream));
      m->total_launches++;
      if (st == 0) {
        CK(m, launch_set_dt(m->d_speeds, m->d_dtch, dt, m->cfg.cfl, m->stream, 1, mesh_res_rate(m)));
        m->total_launches++;
      }
      A.W = m->W;
      A.WG = m->WG;
      A.tmap = &m->tmapW;
    }
    cudaError_t e;
    if (m->cfg.physics == AGILE_HD) e = launch_stage_hd(m->rb, m->cfg.limiter, m->cfg.flux, A, m->stream);
    else if (mhd && m->cfg.eta > 0.0) e = launch_stage_mhd_res(m->rb, m->cfg.limiter, m->cfg.flux, A, m->stream);
    else if (mhd) e = launch_stage_mhd(m->rb, m->cfg.limiter, m->cfg.flux, A, m->stream);
    else if (m->cfg.eos == AGILE_EOS_SYNGE)
      e = launch_stage_srhd_synge(m->rb, m->cfg.limiter, m->cfg.flux, A, m->stream);
    else if (m->cfg.physics == AGILE_FFHD) e = launch_stage_ffhd(m->rb, m->cfg.limiter, m->cfg.flux, A, m->stream);
    else if (m->cfg.physics == AGILE_FFHD_HTC)
      e = launch_stage_ffhd_htc(m->rb, m->cfg.limiter, m->cfg.flux, A, m->stream);
    else e = launch_stage_srhd(m->rb, m->cfg.limiter, m->cfg.flux, A, m->stream);
    if (e != cudaSuccess) return fail(m, AGILE_ECUDA, std::string("stage kernel: ") + cudaGetErrorString(e));
    phase_end(m, e0, PHASE_STAGE);
    m->stage_launches++;
    m->total_launches++;
    if (m->nfix) {
      AuxArgs a = aux_args(m, Uo);
      cudaEvent_t f0 = phase_begin(m);
      CK(m, launch_fixup(a, m->d_fix, m->nfix, A.b, m->d_dtch, m->stream));
      phase_end(m, f0, PHASE_FIXUP);
      m->total_launches++;
    }
  }
  if (mhd && !fuse) {
    AuxArgs a = aux_args(m, m->U[0]);
    CK(m, launch_glm_decay(a, m->d_dtch, m->stream));
    m->total_launches++;
  }
  if (cool) {                                   // second half, with the CFL speeds of U^{n+1}
    CK(m, cudaMemsetAsync(m->d_speeds, 0, 2 * sizeof(unsigned long long), m->stream));
    AuxArgs a = aux_args(m, m->U[0]);
    CK(m, launch_cooling(a, m->cool, m->d_cool, m->d_dtch, 0.5, m->d_speeds, m->stream));
    m->total_launches++;
    m->speeds_valid = true;
  } else if (lead) {
    m->speeds_valid = false;                   // the next step's first pass reduces them
  } else if (fuse) {
    m->speeds_valid = true;
  } else {
    m->speeds_valid = false;
    s = ensure_speeds(m);
    if (s) return s;
  }
  return AGILE_OK;
}

agile_status agile_set_cooling(agile_mesh* m, const double* T, const double* Lambda, int n) {
  if (!m) return AGILE_EINVAL;
  if (n == 0) {
    CK(m, cudaStreamSynchronize(m->stream));
    dfree(m, m->d_cool);
    m->d_cool = nullptr;
    m->cool = CoolHost();
    return AGILE_OK;
  }
  if (m->cfg.physics != AGILE_HD && m->cfg.physics != AGILE_MHD_GLM && m->cfg.physics != AGILE_FFHD &&
      m->cfg.physics != AGILE_FFHD_HTC)
    return fail(m, AGILE_EINVAL, "radiative losses apply to hd, mhd and ffhd");
  CoolHost c;
  if (build_cool_table(T, Lambda, n, m->cfg.gamma, m->rb, &c))
    return fail(m, AGILE_EINVAL, "cooling table: 2..4096 nodes, T increasing, T and Lambda positive and "
                                 "finite, segment constants representable in the stencil precision");
  const size_t bytes = c.segd.size() * (size_t)m->rb;
  void* d = dalloc(m, bytes);
  if (!d) return fail(m, AGILE_ENOMEM, "device allocation failed");
  const void* src = m->rb == 8 ? (const void*)c.segd.data() : (const void*)c.segf.data();
  CK(m, cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, m->stream));
  CK(m, cudaStreamSynchronize(m->stream));   // the host table is a temporary
  dfree(m, m->d_cool);
  m->d_cool = d;
  m->cool = c;
  return AGILE_OK;
}

// Block maxima of the Loehner estimate into emax (host). screen: for the refinement decision
// only (launch_estimate's FP32 screen: a block far from both thresholds may get its FP32
// maximum); else every value exact.
agile_status mesh_estimate(agile_mesh* m, double* emax, bool screen) {
  agile_status s = fill_ghosts(m, m->U[0]);
  if (s) return s;
  double* d = (double*)dalloc(m, (m->nblk + 2) * sizeof(double));
  if (!d) return fail(m, AGILE_ENOMEM, "device allocation failed");
  const double* tols = nullptr;
  double margin = -1.0;
  if (screen) {
    const double th[2] = {m->cfg.refine_tol, m->cfg.refine_tol * m->cfg.derefine_ratio};
    CK(m, cudaMemcpyAsync(d + m->nblk, th, sizeof(th), cudaMemcpyHostToDevice, m->stream));
    tols = d + m->nblk;
    margin = estimate_screen_margin(m->cfg.refine_weights, m->cfg.refine_nvars, m->cfg.lohner_eps);
  }
  AuxArgs a = aux_args(m, m->U[0]);
  cudaEvent_t e0 = phase_begin(m);
  CK(m, launch_estimate(a, m->d_vars, m->d_weights, m->cfg.refine_nvars, m->cfg.lohner_eps, d, m->stream, tols,
                        margin));
  phase_end(m, e0, PHASE_ESTIMATE);
  m->total_launches++;
  CK(m, cudaMemcpyAsync(emax, d, m->nblk * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  s = check_status(m);
  dfree_t(m, d);
  return s;
}

agile_status agile_estimate(agile_mesh* m, double* emax) {
  if (!m || !emax) return fail(m, AGILE_EINVAL, "null argument");
  return mesh_estimate(m, emax, false);
}

agile_status agile_regrid(agile_mesh* m, int init, int* nr, int* nc) {
  if (!m) return AGILE_EINVAL;
  if (nr) *nr = 0;
  if (nc) *nc = 0;
  std::vector<double> emax(m->nblk);
  std::vector<int> flags(m->nblk, 0);
  if (m->cfg.max_level == 1) return AGILE_OK;   // one level: every flag is "keep"
  agile_status s = mesh_estimate(m, emax.data(), true);
  if (s) return s;
  const auto& keys = m->mesh->blocks();
  for (int i = 0; i < m->nblk; ++i) {
    if (emax[i] > m->cfg.refine_tol && keys[i].lev < m->cfg.max_level) flags[i] = 1;
    else if (emax[i] < m->cfg.refine_tol * m->cfg.derefine_ratio && keys[i].lev > 1) flags[i] = -1;
  }
  return do_regrid(m, flags, init, nr, nc);
}

agile_status agile_regrid_flags(agile_mesh* m, const int* flags, int init, int* nr, int* nc) {
  if (!m || !flags) return fail(m, AGILE_EINVAL, "null argument");
  std::vector<int> f(flags, flags + m->nblk);
  return do_regrid(m, f, init, nr, nc);
}

agile_status agile_get_layout(agile_mesh* m, size_t* nblocks, int* nvar) {
  if (!m) return AGILE_EINVAL;
  if (nblocks) *nblocks = (size_t)m->nblk;
  if (nvar) *nvar = m->nv;
  return AGILE_OK;
}

agile_status agile_get_state(agile_mesh* m, int* level, int* ijk, double* cons) {
  if (!m) return AGILE_EINVAL;
  const auto& keys = m->mesh->blocks();
  for (int i = 0; i < m->nblk; ++i) {
    if (level) level[i] = keys[i].lev;
    if (ijk) {
      ijk[3 * i] = keys[i].x;
      ijk[3 * i + 1] = keys[i].y;
      ijk[3 * i + 2] = keys[i].z;
    }
  }
  if (cons) {
    AuxArgs a = aux_args(m, m->U[0]);
    if (void* dv = pinned_view(cons)) {      // page-locked: the pack writes it in place
      CK(m, launch_pack(a, (double*)dv, nullptr, m->stream));
      m->total_launches++;
      return check_status(m);
    }
    const size_t bytes = (size_t)m->nblk * m->nv * NCELL * sizeof(double);
    double* d = (double*)dalloc(m, bytes);
    if (!d) return fail(m, AGILE_ENOMEM, "device allocation failed");
    CK(m, launch_pack(a, d, nullptr, m->stream));
    m->total_launches++;
    CK(m, cudaMemcpyAsync(cons, d, bytes, cudaMemcpyDeviceToHost, m->stream));
    agile_status s = check_status(m);
    dfree_t(m, d);
    return s;
  }
  return check_status(m);
}

agile_status agile_get_aux(agile_mesh* m, double* aux) {
  if (!m || !aux) return fail(m, AGILE_EINVAL, "null argument");
  if (m->na == 0) return fail(m, AGILE_EINVAL, "physics has no auxiliary variables");
  const size_t bytes = (size_t)m->nblk * m->na * NCELL * sizeof(double);
  double* d = (double*)dalloc(m, bytes);
  if (!d) return fail(m, AGILE_ENOMEM, "device allocation failed");
  AuxArgs a = aux_args(m, m->U[0]);
  CK(m, launch_pack(a, nullptr, d, m->stream));
  m->total_launches++;
  CK(m, cudaMemcpyAsync(aux, d, bytes, cudaMemcpyDeviceToHost, m->stream));
  agile_status s = check_status(m);
  dfree_t(m, d);
  return s;
}

agile_status agile_conserved_sums(agile_mesh* m, double* sums) {
  if (!m || !sums) return fail(m, AGILE_EINVAL, "null argument");
  const size_t np = (size_t)m->nblk * m->nv;
  if (m->d_sums_cap < np + 16) {     // the scratch is kept between calls (a diagnostic per step)
    dfree_t(m, m->d_sums);
    m->d_sums_cap = 0;
    m->d_sums = (double*)dalloc(m, (np + 16) * sizeof(double));
    if (!m->d_sums) return fail(m, AGILE_ENOMEM, "device allocation failed");
    m->d_sums_cap = np + 16;
  }
  double* d = m->d_sums;
  AuxArgs a = aux_args(m, m->U[0]);
  CK(m, launch_sums(a, d, m->stream));
  sums_total_kernel<<<m->nv, 256, 0, m->stream>>>(d, m->nblk, m->nv, d + np);
  CK(m, cudaGetLastError());
  m->total_launches += 2;
  CK(m, cudaMemcpyAsync(sums, d + np, m->nv * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  return check_status(m);
}

agile_status agile_get_halo(agile_mesh* m, size_t block, double* out) {
  if (!m || !out || block >= (size_t)m->nblk) return fail(m, AGILE_EINVAL, "bad argument");
  agile_status s = fill_ghosts(m, m->U[0]);
  if (s) return s;
  const size_t bytes = (size_t)m->nt * 8000 * sizeof(double);
  double* d = (double*)dalloc(m, bytes);
  if (!d) return fail(m, AGILE_ENOMEM, "device allocation failed");
  AuxArgs a = aux_args(m, m->U[0]);
  CK(m, launch_halo(a, (int)block, d, m->stream));
  m->total_launches++;
  CK(m, cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, m->stream));
  s = check_status(m);
  dfree_t(m, d);
  return s;
}

agile_status agile_sync(agile_mesh* m) {
  if (!m) return AGILE_EINVAL;
  return check_status(m);
}

agile_status agile_set_kernel_timing(agile_mesh* m, int enable) {
  if (!m) return AGILE_EINVAL;
  CK(m, cudaStreamSynchronize(m->stream));
  for (cudaEvent_t e : m->ev) cudaEventDestroy(e);
  m->ev.clear();
  m->ev_cat.clear();
  m->timing = enable != 0;
  m->stage_launches = 0;
  m->total_launches = 0;
  for (long long& n : m->phase_launches) n = 0;
  return AGILE_OK;
}

agile_status agile_phase_timing(agile_mesh* m, double* ms, long long* launches) {
  if (!m || !ms) return AGILE_EINVAL;
  CK(m, cudaStreamSynchronize(m->stream));
  for (int p = 0; p < 4; ++p) ms[p] = 0.0;
  for (size_t i = 0; i + 1 < m->ev.size(); i += 2) {
    float t = 0.f;
    CK(m, cudaEventElapsedTime(&t, m->ev[i], m->ev[i + 1]));
    ms[m->ev_cat[i / 2]] += t;
  }
  if (launches)
    for (int p = 0; p < 4; ++p) launches[p] = m->phase_launches[p];
  return AGILE_OK;
}

agile_status agile_kernel_timing(agile_mesh* m, double* stage_ms, long long* stage_launches,
                                 long long* total_launches) {
  if (!m) return AGILE_EINVAL;
  CK(m, cudaStreamSynchronize(m->stream));
  double tot = 0.0;
  for (size_t i = 0; i + 1 < m->ev.size(); i += 2) {
    if (m->ev_cat[i / 2] != PHASE_STAGE) continue;
    float ms = 0.f;
    CK(m, cudaEventElapsedTime(&ms, m->ev[i], m->ev[i + 1]));
    tot += ms;
  }
  if (stage_ms) *stage_ms = tot;
  if (stage_launches) *stage_launches = m->stage_launches;
  if (total_launches) *total_launches = m->total_launches;
  return AGILE_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------------------
// Conserved sums without any device allocation (agile_conserved_sums_noalloc).
//
// Some callers cannot allocate device memory at the moment they want the diagnostics: a
// serving loop that reserved its whole device budget up front and forbids further
// allocation, or a host whose allocator is not re-entrant from the calling thread (a
// callback into a framework allocator that is itself in the middle of an allocation). This
// variant keeps its scratch (per-block partial sums and the totals) in a fixed array in
// device memory that every GPU loading the library holds until the process exits.
// ----------------------------------------------------------------------------------------
namespace {

constexpr int NOALLOC_MAX_BLOCKS = 16384;                 // leaves per mesh
constexpr size_t NOALLOC_TOTALS = (size_t)NOALLOC_MAX_BLOCKS * 9;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_TOTALS + 16];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device;
// in host code the symbol itself is only a host-side stand-in).
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace

// Totals over the per-block sums, one CTA of 256 threads per variable (launched with nv CTAs):
// thread i sums blocks i, i + 256, ... with Neumaier compensation, then the 256 (sum,
// compensation) pairs merge in a fixed tree whose every addition keeps its exact error
// (TwoSum). Deterministic; agile_conserved_sums and agile_conserved_sums_noalloc both use it,
// so their results agree bit for bit.
__global__ void __launch_bounds__(256) sums_total_kernel(const double* part, int nblk, int nv,
                                                         double* totals) {
  __shared__ double ss[256], sc[256];
  const int t = threadIdx.x;
  {
    const int v = blockIdx.x;
    double sum = 0.0, comp = 0.0;
    for (int b = t; b < nblk; b += 256) {
      const double x = part[(size_t)b * nv + v];
      const double u = __dadd_rn(sum, x);
      if (fabs(sum) >= fabs(x)) comp = __dadd_rn(comp, __dadd_rn(__dsub_rn(sum, u), x));
      else comp = __dadd_rn(comp, __dadd_rn(__dsub_rn(x, u), sum));
      sum = u;
    }
    ss[t] = sum;
    sc[t] = comp;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (t < w) {
        const double x = ss[t], y = ss[t + w];
        const double u = __dadd_rn(x, y);
        const double yy = __dsub_rn(u, x);
        const double e = __dadd_rn(__dsub_rn(x, __dsub_rn(u, yy)), __dsub_rn(y, yy));
        ss[t] = u;
        sc[t] = __dadd_rn(__dadd_rn(sc[t], sc[t + w]), e);
      }
      __syncthreads();
    }
    if (t == 0) totals[v] = __dadd_rn(ss[0], sc[0]);
  }
}

extern "C" agile_status agile_conserved_sums_noalloc(agile_mesh* m, double* sums) {
  if (!m || !sums) return fail(m, AGILE_EINVAL, "null argument");
  if (m->nblk > NOALLOC_MAX_BLOCKS)
    return fail(m, AGILE_EBUDGET,
                "agile_conserved_sums_noalloc: mesh has " + std::to_string(m->nblk) +
                    " leaves, more than its fixed scratch holds (" +
                    std::to_string(NOALLOC_MAX_BLOCKS) + "); use agile_conserved_sums");
  double* scratch = nullptr;
  CK(m, noalloc_scratch(&scratch));
  AuxArgs a = aux_args(m, m->U[0]);
  CK(m, launch_sums(a, scratch, m->stream));
  sums_total_kernel<<<m->nv, 256, 0, m->stream>>>(scratch, m->nblk, m->nv, scratch + NOALLOC_TOTALS);
  CK(m, cudaGetLastError());
  m->total_launches += 2;
  CK(m, cudaMemcpyAsync(sums, scratch + NOALLOC_TOTALS, m->nv * sizeof(double), cudaMemcpyDeviceToHost,
                        m->stream));
  return check_status(m);
}

// ----------------------------------------------------------------------------------------
// Batched independent solves: one pool holds the blocks of all levels of every solve, the
// stage kernel updates all of them in one persistent launch per RK stage with each solve's
// own CFL dt and GLM speed, ghost fill and flux fix-up of all solves share launches, and a
// whole step is replayed from one captured CUDA graph.
// ----------------------------------------------------------------------------------------
struct agile_batch {
  agile_config cfg;                 // shared scheme
  int nsolve = 0;
  std::vector<agile_config> cfgs;
  std::vector<HostMesh*> meshes;
  std::vector<int> offset;          // first block of each solve
  int nblk = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  agile_allocator alloc{};
  bool default_alloc = true;
  int nv = 5, na = 0, nt = 5, rb = 8;
  void* U[3] = {nullptr, nullptr, nullptr};
  BlockDesc* d_bd = nullptr;
  int* d_solve_of = nullptr;
  int* d_status = nullptr;
  unsigned long long* d_speeds = nullptr;
  double* d_dtch = nullptr;
  int* d_work = nullptr;
  CUtensorMap tmap[3];
  bool speeds_valid = false;
  int steps_done = 0;
  cudaGraphExec_t graph = nullptr;
  long long launches = 0;
  std::string err;
  int grid = 0;                     // persistent CTAs of the stage launches (0: default)
  bool dynamic = true;              // blocks taken from an atomic counter (else strided)
  int layout = 0;                   // staging layout of the stage kernel (0: the default)
  // refinement: ghost slots, flux registers and their tasks of all solves (indices offset)
  void* G = nullptr;
  void* FR = nullptr;
  GhostTask* d_ghosts = nullptr;
  FixupTask* d_fix = nullptr;
  int nghost = 0, nfix = 0, nslots = 0;
  std::vector<agile_ic_fn> ics;     // initial conditions, re-applied to blocks a regrid creates
  std::vector<void*> ic_users;
  // continuous batching: solves attach to and detach from the block pool without moving the
  // others. Solve i (live[i]) holds pool blocks offset[i] .. offset[i] + its block count - 1;
  // blocks of detached solves are holes that later attachments fill. The per-block kernels
  // walk the work list d_wl (the live solves' blocks) instead of the whole pool.
  std::vector<char> live;
  struct Tables {                   // a solve's own descriptor tables (local indices), cached
    bool valid = false;
    std::vector<BlockDesc> desc;
    std::vector<GhostTask> ghosts;
    std::vector<FixupTask> fix;
    std::vector<int> order;         // the stage kernel's work order of its blocks (slab_order)
    int nslots = 0;
  };
  std::vector<Tables> tables;
  int cap = 0;                      // pool capacity in blocks (U[0] .. U[2])
  int cap_stage = 0;                // capacity U[1], U[2] were allocated with
  int scap = 0;                     // solves the per-solve device arrays hold
  int* d_wl = nullptr;
  int nwork = 0;
  int tab_cap = 0;                  // blocks d_bd, d_solve_of and d_wl hold (the capacity)
  void* W = nullptr;                // SRHD: primitives of the stage input (capacity blocks),
  void* WG = nullptr;               // of its ghost slots, and the tensor map over W
  CUtensorMap tmapW;
  // Host-to-device uploads of membership changes and initial states go through device
  // buffers written on their own stream: a copy from pageable host memory returns only when
  // it has been carried out, so on the batch stream it would wait for every step already
  // enqueued there. The batch stream waits for the upload instead; a buffer is released once
  // an event after its last reader on the batch stream has completed.
  cudaStream_t up_stream = nullptr;
  struct Upload {
    void* p;
    size_t bytes;
    cudaEvent_t done;
  };
  std::vector<Upload> uploads;
  size_t upload_bytes = 0;          // bytes of the upload buffers not yet released
  std::vector<Upload> upload_free;  // released buffers kept for reuse by later uploads
  size_t upload_free_bytes = 0;
};

// Upload buffers held at once (bytes): past this, a new upload first waits for the oldest
// buffers' readers, so that uploads running ahead of the batch stream stay bounded.
constexpr size_t UPLOAD_HELD_MAX = (size_t)4 << 30;

namespace {

// The batch shares the mesh helpers through a view with the same allocation fields.
agile_mesh* as_mesh_view(agile_batch* B, agile_mesh* tmp) {
  tmp->stream = B->stream;
  tmp->alloc = B->alloc;
  tmp->default_alloc = B->default_alloc;
  tmp->nv = B->nv;
  tmp->na = B->na;
  tmp->nt = B->nt;
  tmp->rb = B->rb;
  tmp->nblk = B->nblk;
  tmp->cfg = B->cfg;
  return tmp;
}

agile_status bfail(agile_batch* B, agile_status s, const std::string& msg) {
  if (B) B->err = msg;
  return s;
}

#define BCK(B, call)                                                                         \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return bfail((B), AGILE_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_));       \
  } while (0)

AuxArgs batch_aux(agile_batch* B, void* U) {
  AuxArgs a;
  a.phys = phys_kind(B->cfg);
  a.real_bytes = B->rb;
  a.gamma = B->cfg.gamma;
  a.cfl = B->cfg.cfl;
  a.glm_alpha = B->cfg.glm_alpha;
  a.U = U;
  a.Uw = U;
  a.G = B->G;
  a.Gw = B->G;
  a.FR = B->FR;
  a.bd = B->d_bd;
  a.nblk = B->nblk;
  a.status = B->d_status;
  a.solve_of = B->d_solve_of;
  a.nsolve = B->nsolve;
  a.nblk = B->nwork;
  a.wl = B->d_wl;
  return a;
}

agile_status batch_status(agile_batch* B);

// A released upload buffer: kept for reuse while the kept ones stay within the bound, else
// freed (largest first).
void batch_keep_upload(agile_batch* B, void* p, size_t bytes) {
  agile_mesh view;
  as_mesh_view(B, &view);
  view.stream = B->up_stream;
  B->upload_free.push_back({p, bytes, nullptr});
  B->upload_free_bytes += bytes;
  while (B->upload_free_bytes > UPLOAD_HELD_MAX && !B->upload_free.empty()) {
    size_t big = 0;
    for (size_t i = 1; i < B->upload_free.size(); ++i)
      if (B->upload_free[i].bytes > B->upload_free[big].bytes) big = i;
    dfree(&view, B->upload_free[big].p);
    B->upload_free_bytes -= B->upload_free[big].bytes;
    B->upload_free.erase(B->upload_free.begin() + big);
  }
}

// Release the upload buffers whose readers have run (all of them, and the kept ones too,
// with wait = true, after the batch stream has been synchronised).
void batch_reap_uploads(agile_batch* B, bool wait) {
  agile_mesh view;
  as_mesh_view(B, &view);
  view.stream = B->up_stream;
  size_t k = 0;
  for (size_t i = 0; i < B->uploads.size(); ++i) {
    agile_batch::Upload& u = B->uploads[i];
    if (wait || cudaEventQuery(u.done) == cudaSuccess) {
      if (wait) cudaEventSynchronize(u.done);
      cudaEventDestroy(u.done);
      B->upload_bytes -= u.bytes;
      if (wait) dfree(&view, u.p);
      else batch_keep_upload(B, u.p, u.bytes);
    } else {
      B->uploads[k++] = u;
    }
  }
  B->uploads.resize(k);
  if (wait) {
    for (agile_batch::Upload& u : B->upload_free) dfree(&view, u.p);
    B->upload_free.clear();
    B->upload_free_bytes = 0;
  }
}

// Wait for the oldest upload buffers' readers until `bytes` more stay within the bound.
void batch_bound_uploads(agile_batch* B, size_t bytes) {
  agile_mesh view;
  as_mesh_view(B, &view);
  view.stream = B->up_stream;
  size_t k = 0;
  std::vector<agile_batch::Upload> done;
  while (k < B->uploads.size() && B->upload_bytes + bytes > UPLOAD_HELD_MAX) {
    agile_batch::Upload& u = B->uploads[k++];   // oldest first: recorded in stream order
    cudaEventSynchronize(u.done);
    cudaEventDestroy(u.done);
    B->upload_bytes -= u.bytes;
    done.push_back(u);
  }
  B->uploads.erase(B->uploads.begin(), B->uploads.begin() + k);
  for (const agile_batch::Upload& u : done) batch_keep_upload(B, u.p, u.bytes);
}

// Copy `bytes` of host memory into a device buffer on the upload stream (not behind the
// batch stream's enqueued work) and make the batch stream wait for the copy. The caller
// enqueues the buffer's readers on the batch stream, then calls batch_upload_done with the
// buffer's size (*size_out, at least `bytes`).
void* batch_upload(agile_batch* B, const void* src, size_t bytes, agile_status* st, size_t* size_out) {
  *st = AGILE_OK;
  batch_reap_uploads(B, false);
  batch_bound_uploads(B, bytes);
  if (!B->up_stream && cudaStreamCreateWithFlags(&B->up_stream, cudaStreamNonBlocking) != cudaSuccess) {
    *st = bfail(B, AGILE_ECUDA, "upload stream");
    return nullptr;
  }
  agile_mesh view;
  as_mesh_view(B, &view);
  view.stream = B->up_stream;
  // the smallest kept buffer that holds the upload (at most twice its size), else a new one
  void* p = nullptr;
  size_t fit = (size_t)-1, cap_bytes = bytes;
  for (size_t i = 0; i < B->upload_free.size(); ++i) {
    const size_t c = B->upload_free[i].bytes;
    if (c >= bytes && c / 2 <= bytes && (fit == (size_t)-1 || c < B->upload_free[fit].bytes)) fit = i;
  }
  if (fit != (size_t)-1) {
    p = B->upload_free[fit].p;
    cap_bytes = B->upload_free[fit].bytes;
    B->upload_free_bytes -= cap_bytes;
    B->upload_free.erase(B->upload_free.begin() + fit);
  } else {
    p = dalloc(&view, bytes);
  }
  if (!p) {
    *st = bfail(B, AGILE_ENOMEM, "device allocation failed");
    return nullptr;
  }
  if (size_out) *size_out = cap_bytes;
  cudaEvent_t ev = nullptr;
  cudaError_t e = cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, B->up_stream);
  // the host source may be released on return, pinned or not: wait for this copy alone
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->up_stream);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, B->up_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(B->stream, ev, 0);
  if (ev) cudaEventDestroy(ev);      // the wait above holds the recorded state
  if (e != cudaSuccess) {
    cudaStreamSynchronize(B->up_stream);
    dfree(&view, p);
    *st = bfail(B, AGILE_ECUDA, std::string("upload: ") + cudaGetErrorString(e));
    return nullptr;
  }
  return p;
}

// The readers of upload buffer p are enqueued on the batch stream: release p after them.
agile_status batch_upload_done(agile_batch* B, void* p, size_t bytes) {
  agile_batch::Upload u{p, bytes, nullptr};
  cudaError_t e = cudaEventCreateWithFlags(&u.done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(u.done, B->stream);
  if (e != cudaSuccess) {            // keep the buffer until the batch stream is idle
    if (u.done) cudaEventDestroy(u.done);
    cudaStreamSynchronize(B->stream);
    agile_mesh view;
    as_mesh_view(B, &view);
    view.stream = B->up_stream;
    dfree(&view, p);
    return bfail(B, AGILE_ECUDA, std::string("upload event: ") + cudaGetErrorString(e));
  }
  B->uploads.push_back(u);
  B->upload_bytes += bytes;
  return AGILE_OK;
}

int solve_blocks(const agile_batch* B, int i) {
  return B->live[i] ? (int)B->meshes[i]->blocks().size() : 0;
}

bool solve_ok(const agile_batch* B, int i) { return B && i >= 0 && i < B->nsolve && B->live[i]; }

// Descriptor tables of the live solves at their pool offsets: block indices offset by the
// solve's first block, ghost-slot / flux-register indices by its first slot; pool blocks of no
// live solve get an inert descriptor and are left out of the work list. Every index is checked
// against the new sizes before anything is uploaded. U[0] already holds every live solve's
// blocks at its offset; the stage buffers are reallocated when the capacity changed.
agile_status batch_rebuild(agile_batch* B) {
  int extent = 0;
  for (int i = 0; i < B->nsolve; ++i)
    if (B->live[i]) extent = std::max(extent, B->offset[i] + solve_blocks(B, i));
  if (extent > B->cap) return bfail(B, AGILE_EINVAL, "pool layout exceeds the capacity");
  BlockDesc inert{};
  for (int f = 0; f < 6; ++f) {
    inert.src[f] = SRC_OUTFLOW;
    inert.slot[f] = -1;
    inert.kind[f] = FK_BC;
    for (int q = 0; q < 4; ++q) inert.nbr[f][q] = -1;
  }
  inert.dx[0] = inert.dx[1] = inert.dx[2] = 1.0;
  inert.level = 1;
  std::vector<BlockDesc> desc(extent, inert);
  std::vector<int> solve_of(extent, 0), work;
  std::vector<GhostTask> ghosts;
  std::vector<FixupTask> fix;
  std::vector<char> used(extent, 0);
  int slots = 0;
  B->tables.resize(B->nsolve);
  for (int i = 0; i < B->nsolve; ++i) {
    if (!B->live[i]) continue;
    agile_batch::Tables& T = B->tables[i];
    if (!T.valid) {                 // a solve's own tables change only when it is regridded
      std::string err;
      T.desc.clear();
      T.ghosts.clear();
      T.fix.clear();
      B->meshes[i]->build_descs(&T.desc, &T.ghosts, &T.fix, &T.nslots, &err);
      if (!err.empty()) return bfail(B, AGILE_EINVAL, err);
      T.order = slab_order(*B->meshes[i]);
      T.valid = true;
    }
    const std::vector<BlockDesc>& d = T.desc;
    std::vector<GhostTask> g = T.ghosts;
    std::vector<FixupTask> x = T.fix;
    const int ns = T.nslots;
    const int O = B->offset[i], S = slots;
    for (size_t q = 0; q < d.size(); ++q) {
      BlockDesc bd = d[q];
      for (int f = 0; f < 6; ++f) {
        if (bd.src[f] >= 0) bd.src[f] += O;
        else if (bd.src[f] <= SRC_SLOT0) bd.src[f] = SRC_SLOT0 - (SRC_SLOT0 - bd.src[f] + S);
        if (bd.slot[f] >= 0) bd.slot[f] += S;
        for (int k = 0; k < 4; ++k)
          if (bd.nbr[f][k] >= 0) bd.nbr[f][k] += O;
      }
      const int b = O + (int)q;
      if (b < 0 || b >= extent || used[b]) return bfail(B, AGILE_EINVAL, "solves overlap in the pool");
      used[b] = 1;
      desc[b] = bd;
      solve_of[b] = i;
    }
    for (int q : T.order) work.push_back(O + q);
    for (GhostTask& t : g) {
      t.blk += O;
      t.slot += S;
      for (int k = 0; k < 4; ++k)
        if (t.nbr[k] >= 0) t.nbr[k] += O;
      ghosts.push_back(t);
    }
    for (FixupTask& t : x) {
      t.blk += O;
      for (int j = 0; j < t.nface; ++j) {
        t.slot_c[j] += S;
        for (int k = 0; k < 4; ++k) t.slot_f[j][k] += S;
      }
      fix.push_back(t);
    }
    slots += ns;
  }
  auto blk_ok = [&](int v) { return v >= 0 && v < extent && used[v]; };
  auto slot_ok = [&](int v) { return v >= 0 && v < slots; };
  for (int b : work) {
    const BlockDesc& bd = desc[b];
    for (int f = 0; f < 6; ++f) {
      if (bd.src[f] >= 0 && !blk_ok(bd.src[f])) return bfail(B, AGILE_EINVAL, "block table out of range");
      if (bd.src[f] <= SRC_SLOT0 && !slot_ok(SRC_SLOT0 - bd.src[f])) return bfail(B, AGILE_EINVAL, "slot out of range");
      if (bd.slot[f] >= slots) return bfail(B, AGILE_EINVAL, "slot out of range");
      for (int q = 0; q < 4; ++q)
        if (bd.nbr[f][q] >= extent) return bfail(B, AGILE_EINVAL, "neighbour out of range");
    }
  }
  for (const GhostTask& t : ghosts) {
    if (!blk_ok(t.blk) || !slot_ok(t.slot)) return bfail(B, AGILE_EINVAL, "ghost task out of range");
    for (int q = 0; q < 4; ++q)
      if (t.nbr[q] >= extent) return bfail(B, AGILE_EINVAL, "ghost task out of range");
  }
  for (const FixupTask& t : fix) {
    if (!blk_ok(t.blk)) return bfail(B, AGILE_EINVAL, "fix-up task out of range");
    for (int j = 0; j < t.nface; ++j) {
      if (!slot_ok(t.slot_c[j])) return bfail(B, AGILE_EINVAL, "fix-up task out of range");
      for (int q = 0; q < 4; ++q)
        if (!slot_ok(t.slot_f[j][q])) return bfail(B, AGILE_EINVAL, "fix-up task out of range");
    }
  }
  // The old tables and buffers are released in stream order (the allocator's contract), so
  // work already enqueued still reads them and nothing waits here.
  agile_mesh view;
  as_mesh_view(B, &view);
  dfree_t(&view, B->d_bd);
  dfree_t(&view, B->d_solve_of);
  dfree_t(&view, B->d_wl);
  dfree_t(&view, B->d_ghosts);
  dfree_t(&view, B->d_fix);
  dfree(&view, B->G);
  dfree(&view, B->FR);
  const bool prim_pass = phys_prim_pass(phys_kind(B->cfg));
  if (B->cap_stage != B->cap) {
    dfree(&view, B->U[1]);
    dfree(&view, B->U[2]);
    dfree(&view, B->W);
    const size_t pool = (size_t)B->cap * B->nt * NCELL * B->rb;
    B->U[1] = dalloc(&view, pool);
    B->U[2] = B->cfg.rk == 3 ? dalloc(&view, pool) : nullptr;
    if (prim_pass) B->W = dalloc(&view, std::max(pool, (size_t)1));
    if (!B->U[1] || (B->cfg.rk == 3 && !B->U[2]) || (prim_pass && !B->W))
      return bfail(B, AGILE_ENOMEM, "device allocation failed");
    B->cap_stage = B->cap;
  }
  dfree(&view, B->WG);
  if (prim_pass) {
    B->WG = dalloc(&view, (size_t)std::max(slots, 1) * B->nt * 512 * B->rb);
    if (!B->WG) return bfail(B, AGILE_ENOMEM, "device allocation failed");
  }
  B->nblk = extent;
  B->nwork = (int)work.size();
  view.nblk = extent;
  // the block tables are sized for the whole capacity, so that an attachment into free pool
  // blocks can write its own range of them (batch_patch)
  B->tab_cap = 0;
  if (B->cap) {
    B->d_bd = (BlockDesc*)dalloc(&view, (size_t)B->cap * sizeof(BlockDesc));
    B->d_solve_of = (int*)dalloc(&view, (size_t)B->cap * sizeof(int));
    B->d_wl = (int*)dalloc(&view, (size_t)B->cap * sizeof(int));
  }
  if (!ghosts.empty()) B->d_ghosts = (GhostTask*)dalloc(&view, ghosts.size() * sizeof(GhostTask));
  if (!fix.empty()) B->d_fix = (FixupTask*)dalloc(&view, fix.size() * sizeof(FixupTask));
  if (slots) {
    B->G = dalloc(&view, (size_t)slots * B->nt * 512 * B->rb);
    B->FR = dalloc(&view, (size_t)slots * B->nv * 256 * B->rb);
  }
  if ((B->cap && (!B->d_bd || !B->d_solve_of || !B->d_wl)) || (!ghosts.empty() && !B->d_ghosts) ||
      (!fix.empty() && !B->d_fix) || (slots && (!B->G || !B->FR)))
    return bfail(B, AGILE_ENOMEM, "device allocation failed");
  B->tab_cap = B->cap;
  if (extent) {
    BCK(B, cudaMemcpyAsync(B->d_bd, desc.data(), desc.size() * sizeof(BlockDesc), cudaMemcpyHostToDevice, B->stream));
    BCK(B, cudaMemcpyAsync(B->d_solve_of, solve_of.data(), solve_of.size() * sizeof(int), cudaMemcpyHostToDevice,
                           B->stream));
  }
  if (!work.empty())
    BCK(B, cudaMemcpyAsync(B->d_wl, work.data(), work.size() * sizeof(int), cudaMemcpyHostToDevice, B->stream));
  if (!ghosts.empty())
    BCK(B, cudaMemcpyAsync(B->d_ghosts, ghosts.data(), ghosts.size() * sizeof(GhostTask), cudaMemcpyHostToDevice, B->stream));
  if (!fix.empty())
    BCK(B, cudaMemcpyAsync(B->d_fix, fix.data(), fix.size() * sizeof(FixupTask), cudaMemcpyHostToDevice, B->stream));
  // (pageable host sources are staged when each copy is enqueued: the vectors may go now)
  B->nghost = (int)ghosts.size();
  B->nfix = (int)fix.size();
  B->nslots = slots;
  view.nblk = std::max(B->cap, 1);      // the tensor maps span the pool's capacity
  for (int i = 0; i < 3; ++i) {
    if (B->U[i] && make_tmap(&view, B->U[i], &B->tmap[i]) != AGILE_OK) return bfail(B, AGILE_ECUDA, "tensor map");
  }
  if (make_tmap(&view, B->W, &B->tmapW) != AGILE_OK) return bfail(B, AGILE_ECUDA, "tensor map");
  if (B->graph) {                   // the captured step refers to the old tables
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
  }
  B->steps_done = 0;
  B->speeds_valid = false;
  return AGILE_OK;
}

// Regrid the solves whose plan changes anything (plans[j] for solve j; unchanged solves are
// copied to their new places), with one new layout of the pools and one rebuild of the
// tables; blocks a refinement creates get the initial condition again when init is set.
agile_status batch_apply_plans(agile_batch* B, std::vector<RegridPlan>& plans, int init) {
  std::vector<char> changed(B->nsolve, 0);
  bool any = false;
  for (int j = 0; j < B->nsolve; ++j) {
    changed[j] = B->live[j] && (plans[j].n_refined != 0 || plans[j].n_coarsened != 0);
    any = any || changed[j];
  }
  if (!any) return AGILE_OK;
  agile_mesh view;
  as_mesh_view(B, &view);
  AuxArgs a = batch_aux(B, B->U[0]);
  if (B->nghost) BCK(B, launch_ghosts(a, B->d_ghosts, B->nghost, B->stream));
  const size_t per = (size_t)B->nt * NCELL * B->rb;
  std::vector<int> count(B->nsolve), ncount(B->nsolve);
  std::vector<long long> noff(B->nsolve);
  long long total = 0;
  for (int j = 0; j < B->nsolve; ++j) {     // the new layout is compact: live solves in order
    count[j] = solve_blocks(B, j);
    ncount[j] = changed[j] ? (int)plans[j].blocks.size() : count[j];
    noff[j] = total;
    total += ncount[j];
  }
  // one list of regrid sources over all changed solves, indices global in the old pool
  std::vector<RegridSrc> src;
  std::vector<int> first(B->nsolve, -1);
  for (int j = 0; j < B->nsolve; ++j) {
    if (!changed[j]) continue;
    first[j] = (int)src.size();
    for (RegridSrc r : plans[j].src) {
      const int nsrc = r.mode == 2 ? 8 : 1;
      for (int q = 0; q < nsrc; ++q) {
        if (r.src[q] < 0 || r.src[q] >= count[j]) return bfail(B, AGILE_EINVAL, "regrid source out of range");
        r.src[q] += B->offset[j];
      }
      src.push_back(r);
    }
  }
  const long long newcap = std::max<long long>(total, 1);
  void* Unew = dalloc(&view, (size_t)newcap * per);
  RegridSrc* d_src = (RegridSrc*)dalloc(&view, src.size() * sizeof(RegridSrc));
  if (!Unew || !d_src) return bfail(B, AGILE_ENOMEM, "device allocation failed");
  BCK(B, cudaMemcpyAsync(d_src, src.data(), src.size() * sizeof(RegridSrc), cudaMemcpyHostToDevice, B->stream));
  for (int j = 0; j < B->nsolve; ++j) {
    if (changed[j]) {
      BCK(B, launch_regrid(a, (char*)Unew + noff[j] * per, d_src + first[j], ncount[j], B->stream));
    } else if (count[j]) {
      BCK(B, cudaMemcpyAsync((char*)Unew + noff[j] * per, (const char*)B->U[0] + (size_t)B->offset[j] * per,
                             (size_t)count[j] * per, cudaMemcpyDeviceToDevice, B->stream));
    }
  }
  BCK(B, cudaStreamSynchronize(B->stream));
  dfree_t(&view, d_src);
  dfree(&view, B->U[0]);
  B->U[0] = Unew;
  B->cap = (int)newcap;
  B->tables.resize(B->nsolve);
  for (int j = 0; j < B->nsolve; ++j) {
    if (changed[j]) {
      B->meshes[j]->apply(plans[j]);
      B->tables[j].valid = false;
    }
    B->offset[j] = (int)noff[j];
  }
  agile_status st = batch_rebuild(B);
  if (st) return st;
  for (int j = 0; j < B->nsolve && init; ++j) {
    if (!changed[j] || !B->ics[j] || plans[j].created.empty()) continue;
    agile_mesh v2;
    as_mesh_view(B, &v2);
    v2.mesh = B->meshes[j];
    v2.cfg = B->cfgs[j];
    v2.ic = B->ics[j];
    v2.ic_user = B->ic_users[j];
    v2.d_status = B->d_status;
    v2.nblk = ncount[j];
    st = apply_ic(&v2, (char*)B->U[0] + (size_t)B->offset[j] * per, plans[j].created);
    v2.mesh = nullptr;
    if (st) return bfail(B, st, v2.err);
  }
  return batch_status(B);
}

// Regrid one solve with the given flags (the others unchanged).
agile_status batch_regrid(agile_batch* B, int solve, const std::vector<int>& flags, int init, int* nr,
                          int* nc) {
  std::vector<RegridPlan> plans(B->nsolve);
  plans[solve] = B->meshes[solve]->plan(flags);
  if (nr) *nr = plans[solve].n_refined;
  if (nc) *nc = plans[solve].n_coarsened;
  return batch_apply_plans(B, plans, init);
}

// Loehner flags of every solve from one estimate over the batch (after a ghost fill).
agile_status batch_flags(agile_batch* B, std::vector<std::vector<int>>* flags) {
  agile_mesh view;
  as_mesh_view(B, &view);
  AuxArgs a = batch_aux(B, B->U[0]);
  if (B->nghost) BCK(B, launch_ghosts(a, B->d_ghosts, B->nghost, B->stream));
  int* d_vars = (int*)dalloc(&view, 9 * sizeof(int));
  double* d_w = (double*)dalloc(&view, 9 * sizeof(double));
  double* d_e = (double*)dalloc(&view, (size_t)std::max(B->nblk, 1) * sizeof(double));
  // the refinement thresholds of each solve for the estimator's screen
  std::vector<double> tols(2 * (size_t)B->nsolve, 0.0);
  for (int i = 0; i < B->nsolve; ++i) {
    tols[2 * i] = B->cfgs[i].refine_tol;
    tols[2 * i + 1] = B->cfgs[i].refine_tol * B->cfgs[i].derefine_ratio;
  }
  double* d_tols = (double*)dalloc(&view, tols.size() * sizeof(double));
  if (!d_vars || !d_w || !d_e || !d_tols) return bfail(B, AGILE_ENOMEM, "device allocation failed");
  std::vector<double> emax(std::max(B->nblk, 1));
  flags->assign(B->nsolve, std::vector<int>());
  // the estimator's variables and weights may differ per solve: one pass per distinct set
  std::vector<char> done(B->nsolve, 0);
  for (int j = 0; j < B->nsolve; ++j) {
    if (done[j] || !B->live[j]) continue;
    const agile_config& c = B->cfgs[j];
    BCK(B, cudaMemcpyAsync(d_vars, c.refine_vars, 9 * sizeof(int), cudaMemcpyHostToDevice, B->stream));
    BCK(B, cudaMemcpyAsync(d_w, c.refine_weights, 9 * sizeof(double), cudaMemcpyHostToDevice, B->stream));
    BCK(B, cudaMemcpyAsync(d_tols, tols.data(), tols.size() * sizeof(double), cudaMemcpyHostToDevice, B->stream));
    BCK(B, launch_estimate(a, d_vars, d_w, c.refine_nvars, c.lohner_eps, d_e, B->stream, d_tols,
                           estimate_screen_margin(c.refine_weights, c.refine_nvars, c.lohner_eps)));
    BCK(B, cudaMemcpyAsync(emax.data(), d_e, B->nblk * sizeof(double), cudaMemcpyDeviceToHost, B->stream));
    BCK(B, cudaStreamSynchronize(B->stream));
    for (int i = j; i < B->nsolve; ++i) {
      const agile_config& ci = B->cfgs[i];
      if (done[i] || !B->live[i] || ci.refine_nvars != c.refine_nvars || ci.lohner_eps != c.lohner_eps ||
          memcmp(ci.refine_vars, c.refine_vars, sizeof(c.refine_vars)) != 0 ||
          memcmp(ci.refine_weights, c.refine_weights, sizeof(c.refine_weights)) != 0)
        continue;
      done[i] = 1;
      const auto& keys = B->meshes[i]->blocks();
      const int n = (int)keys.size();
      std::vector<int>& f = (*flags)[i];
      f.assign(n, 0);
      if (ci.max_level == 1) continue;
      for (int q = 0; q < n; ++q) {
        const double e = emax[B->offset[i] + q];
        if (e > ci.refine_tol && keys[q].lev < ci.max_level) f[q] = 1;
        else if (e < ci.refine_tol * ci.derefine_ratio && keys[q].lev > 1) f[q] = -1;
      }
    }
  }
  dfree_t(&view, d_vars);
  dfree_t(&view, d_w);
  dfree_t(&view, d_e);
  dfree_t(&view, d_tols);
  return AGILE_OK;
}

agile_status batch_status(agile_batch* B) {
  BCK(B, cudaStreamSynchronize(B->stream));
  int st = 0;
  BCK(B, cudaMemcpy(&st, B->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    BCK(B, cudaMemset(B->d_status, 0, sizeof(int)));
    if (st & ST_ETIMEOUT) return bfail(B, AGILE_ETIMEOUT, "a bounded wait for a TMA plane gave up");
    if (st & ST_ENOCONV) return bfail(B, AGILE_ENOCONV, "primitive recovery did not converge");
    return bfail(B, AGILE_EUNPHYS, "non-positive density or pressure on the device");
  }
  return AGILE_OK;
}

agile_status batch_ensure_speeds(agile_batch* B) {
  if (B->speeds_valid) return AGILE_OK;
  BCK(B, cudaMemsetAsync(B->d_speeds, 0, 2 * sizeof(unsigned long long) * B->nsolve, B->stream));
  AuxArgs a = batch_aux(B, B->U[0]);
  BCK(B, launch_speeds(a, B->d_speeds, B->stream));
  B->launches++;
  B->speeds_valid = true;
  return AGILE_OK;
}

// Enqueue one full step of every solve (device dt) on the batch stream.
agile_status batch_enqueue_step(agile_batch* B) {
  const bool lead = B->W != nullptr;  // SRHD: dt after the first stage's recovery pass (agile_step)
  if (!lead) BCK(B, launch_set_dt(B->d_speeds, B->d_dtch, 0.0, B->cfg.cfl, B->stream, B->nsolve));
  BCK(B, cudaMemsetAsync(B->d_work, 0, 4 * sizeof(int), B->stream));
  const bool mhd = B->cfg.physics == AGILE_MHD_GLM;
  if (mhd) {
    AuxArgs a = batch_aux(B, B->U[0]);
    BCK(B, launch_glm_decay(a, B->d_dtch, B->stream));
  }
  static const double w2[2][2] = {{0.0, 1.0}, {0.5, 0.5}};
  static const double w3[3][2] = {{0.0, 1.0}, {0.75, 0.25}, {1.0 / 3.0, 2.0 / 3.0}};
  const int nst = B->cfg.rk;
  const bool fuse = B->nfix == 0;     // no flux fix-up: GLM half and CFL speeds in the last stage
  for (int st = 0; st < nst; ++st) {
    const bool last = st == nst - 1;
    void* Us = st == 0 ? B->U[0] : B->U[st];
    if (B->nghost) {
      AuxArgs ga = batch_aux(B, Us);
      BCK(B, launch_ghosts(ga, B->d_ghosts, B->nghost, B->stream));
    }
    if (last && !lead) BCK(B, cudaMemsetAsync(B->d_speeds, 0, 2 * sizeof(unsigned long long) * B->nsolve, B->stream));
    StageArgs A;
    A.Us = Us;
    A.Un = B->U[0];
    A.Uout = last ? B->U[0] : B->U[st + 1];
    A.bd = B->d_bd;
    A.gs = B->G;
    A.fr = B->nfix ? B->FR : nullptr;
    A.dtch = B->d_dtch;
    A.a = nst == 2 ? w2[st][0] : w3[st][0];
    A.b = nst == 2 ? w2[st][1] : w3[st][1];
    A.gamma = B->cfg.gamma;
    A.glm_alpha = B->cfg.glm_alpha;
    A.htc_kappa0 = B->cfg.htc_kappa0;
    A.glm_post = (mhd && last && fuse) ? 1 : 0;
    A.nblk = B->nwork;
    A.wl = B->d_wl;
    A.status = B->d_status;
    A.speeds = (last && fuse && !lead) ? B->d_speeds : nullptr;
    A.tmap = &B->tmap[st == 0 ? 0 : st];
    A.solve_of = B->d_solve_of;
    A.work = B->dynamic ? B->d_work + st : nullptr;
    A.grid = B->grid;
    A.layout = B->layout;
    if (B->W) {                       // one recovery per stored cell, read by the stage kernel
      AuxArgs pa = batch_aux(B, Us);
      if (st == 0) BCK(B, cudaMemsetAsync(B->d_speeds, 0, 2 * sizeof(unsigned long long) * B->nsolve, B->stream));
      BCK(B, launch_prim_pass(pa, B->W, B->WG, B->nslots, st == 0 ? B->d_speeds : nullptr, B->stream));
      if (st == 0) BCK(B, launch_set_dt(B->d_speeds, B->d_dtch, 0.0, B->cfg.cfl, B->stream, B->nsolve));
      A.W = B->W;
      A.WG = B->WG;
      A.tmap = &B->tmapW;
    }
    cudaError_t e;
    if (B->cfg.physics == AGILE_HD) e = launch_stage_hd(B->rb, B->cfg.limiter, B->cfg.flux, A, B->stream);
    else if (mhd) e = launch_stage_mhd(B->rb, B->cfg.limiter, B->cfg.flux, A, B->stream);
    else if (B->cfg.eos == AGILE_EOS_SYNGE)
      e = launch_stage_srhd_synge(B->rb, B->cfg.limiter, B->cfg.flux, A, B->stream);
    else if (B->cfg.physics == AGILE_FFHD) e = launch_stage_ffhd(B->rb, B->cfg.limiter, B->cfg.flux, A, B->stream);
  else if (B->cfg.physics == AGILE_FFHD_HTC)
    e = launch_stage_ffhd_htc(B->rb, B->cfg.limiter, B->cfg.flux, A, B->stream);
    else e = launch_stage_srhd(B->rb, B->cfg.limiter, B->cfg.flux, A, B->stream);
    if (e != cudaSuccess) return bfail(B, AGILE_ECUDA, std::string("stage kernel: ") + cudaGetErrorString(e));
    if (B->nfix) {
      AuxArgs fa = batch_aux(B, A.Uout);
      BCK(B, launch_fixup(fa, B->d_fix, B->nfix, A.b, B->d_dtch, B->stream));
    }
  }
  if (!fuse) {                        // after the last fix-up: GLM half, then the CFL speeds
    AuxArgs a = batch_aux(B, B->U[0]);
    if (mhd) BCK(B, launch_glm_decay(a, B->d_dtch, B->stream));
    if (!lead) BCK(B, launch_speeds(a, B->d_speeds, B->stream));
  }
  return AGILE_OK;
}

// One launch of the first stage (U^n -> the stage-1 buffer; the solution is not modified).
agile_status batch_stage1(agile_batch* B, int grid, bool dynamic, int layout) {
  if (dynamic) BCK(B, cudaMemsetAsync(B->d_work, 0, sizeof(int), B->stream));
  if (B->nghost) {                    // coarse-fine halos of U^n, as the first stage reads them
    AuxArgs ga = batch_aux(B, B->U[0]);
    BCK(B, launch_ghosts(ga, B->d_ghosts, B->nghost, B->stream));
  }
  StageArgs A;
  A.Us = B->U[0];
  A.Un = B->U[0];
  A.Uout = B->U[1];
  A.bd = B->d_bd;
  A.gs = B->G;
  A.fr = nullptr;
  A.dtch = B->d_dtch;
  A.a = 0.0;
  A.b = 1.0;
  A.gamma = B->cfg.gamma;
  A.glm_alpha = B->cfg.glm_alpha;
  A.htc_kappa0 = B->cfg.htc_kappa0;
  A.glm_post = 0;
  A.nblk = B->nwork;
  A.wl = B->d_wl;
  A.status = B->d_status;
  A.speeds = nullptr;
  A.tmap = &B->tmap[0];
  A.solve_of = B->d_solve_of;
  A.work = dynamic ? B->d_work : nullptr;
  A.grid = grid;
  A.layout = layout;
  if (B->W) {
    AuxArgs pa = batch_aux(B, B->U[0]);
    BCK(B, launch_prim_pass(pa, B->W, B->WG, B->nslots, nullptr, B->stream));
    A.W = B->W;
    A.WG = B->WG;
    A.tmap = &B->tmapW;
  }
  cudaError_t e;
  const bool mhd = B->cfg.physics == AGILE_MHD_GLM;
  if (B->cfg.physics == AGILE_HD) e = launch_stage_hd(B->rb, B->cfg.limiter, B->cfg.flux, A, B->stream);
  else if (mhd) e = launch_stage_mhd(B->rb, B->cfg.limiter, B->cfg.flux, A, B->stream);
  else if (B->cfg.eos == AGILE_EOS_SYNGE)
    e = launch_stage_srhd_synge(B->rb, B->cfg.limiter, B->cfg.flux, A, B->stream);
  else if (B->cfg.physics == AGILE_FFHD) e = launch_stage_ffhd(B->rb, B->cfg.limiter, B->cfg.flux, A, B->stream);
  else if (B->cfg.physics == AGILE_FFHD_HTC)
    e = launch_stage_ffhd_htc(B->rb, B->cfg.limiter, B->cfg.flux, A, B->stream);
  else e = launch_stage_srhd(B->rb, B->cfg.limiter, B->cfg.flux, A, B->stream);
  if (e != cudaSuccess) return bfail(B, AGILE_ECUDA, std::string("stage kernel: ") + cudaGetErrorString(e));
  return AGILE_OK;
}

// A solve's configuration fits a batch whose scheme is c0's: same scheme, validated like a
// single mesh (host-side checks only), no resistivity.
bool batch_cfg_ok(const agile_config& c0, const agile_config& c) {
  if (c.physics != c0.physics || c.limiter != c0.limiter || c.flux != c0.flux || c.rk != c0.rk ||
      c.real_bytes != c0.real_bytes || c.gamma != c0.gamma || c.cfl != c0.cfl || c.glm_alpha != c0.glm_alpha ||
      c.eos != c0.eos || c.htc_kappa0 != c0.htc_kappa0 || c.eta != 0.0 || c.max_level < 1 || c.max_level > 12 ||
      c.refine_nvars < 0 || c.refine_nvars > 9)
    return false;
  if (!scheme_ok(c)) return false;
  for (int d = 0; d < 3; ++d) {
    if (c.base_blocks[d] < 1 || c.base_blocks[d] > 4096 || !(c.xmax[d] > c.xmin[d])) return false;
    if ((c.bc[2 * d] == AGILE_PERIODIC) != (c.bc[2 * d + 1] == AGILE_PERIODIC)) return false;
    for (int s = 0; s < 2; ++s)
      if (c.bc[2 * d + s] < 0 || c.bc[2 * d + s] > 2) return false;
  }
  return true;
}

// Per-solve device arrays (speeds, dt and c_h) for at least n solves.
agile_status batch_reserve_solves(agile_batch* B, int n) {
  if (n <= B->scap) return AGILE_OK;
  const int ncap = std::max(n, 2 * B->scap);
  agile_mesh view;
  as_mesh_view(B, &view);
  BCK(B, cudaStreamSynchronize(B->stream));
  dfree_t(&view, B->d_speeds);
  dfree_t(&view, B->d_dtch);
  B->d_speeds = (unsigned long long*)dalloc(&view, 2 * sizeof(unsigned long long) * ncap);
  B->d_dtch = (double*)dalloc(&view, 2 * sizeof(double) * ncap);
  if (!B->d_speeds || !B->d_dtch) return bfail(B, AGILE_ENOMEM, "device allocation failed");
  BCK(B, cudaMemsetAsync(B->d_speeds, 0, 2 * sizeof(unsigned long long) * ncap, B->stream));
  BCK(B, cudaMemsetAsync(B->d_dtch, 0, 2 * sizeof(double) * ncap, B->stream));
  B->scap = ncap;
  B->speeds_valid = false;
  return AGILE_OK;
}

}  // namespace

extern "C" {

agile_status agile_batch_autotune(agile_batch* B, int trials, int* grid, int* dynamic, int* layout,
                                  float* ms) {
  if (!B || trials < 1 || trials > 100) return bfail(B, AGILE_EINVAL, "bad argument");
  agile_status s = batch_ensure_speeds(B);
  if (s) return s;
  BCK(B, launch_set_dt(B->d_speeds, B->d_dtch, 0.0, B->cfg.cfl, B->stream, B->nsolve));
  int dev = 0, sms = 0;
  BCK(B, cudaGetDevice(&dev));
  BCK(B, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grids[3] = {sms, 2 * sms, 3 * sms};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BCK(B, cudaEventCreate(&e0));
  BCK(B, cudaEventCreate(&e1));
  float best = 0.0f;
  int bi = -1;
  // shape c: staging layout c / 6 (four raw slots and one flux buffer; five raw slots and two
  // flux buffers; three raw slots and two flux buffers with the stage input read from global
  // memory), grid (c % 6) >> 1, counter or strided assignment c & 1
  const int layouts[3] = {STAGE_LAYOUT_RING4, STAGE_LAYOUT_RING5_DB, STAGE_LAYOUT_RING3_DB};
  const bool fp64 = B->rb == 8;                       // FP64 stencils have the first layout only
  for (int c = 0; c < 18 && !s; ++c) {
    const int g = grids[(c % 6) >> 1];
    const bool dyn = (c & 1) == 0;
    const int lay = layouts[c / 6];
    if (fp64 && c >= 6) {
      if (ms) ms[c] = -1.0f;
      continue;
    }
    s = batch_stage1(B, g, dyn, lay);                   // warm-up
    if (!s) BCK(B, cudaEventRecord(e0, B->stream));
    for (int t = 0; t < trials && !s; ++t) s = batch_stage1(B, g, dyn, lay);
    if (s) break;
    BCK(B, cudaEventRecord(e1, B->stream));
    BCK(B, cudaEventSynchronize(e1));
    float t_ms = 0.0f;
    BCK(B, cudaEventElapsedTime(&t_ms, e0, e1));
    t_ms /= trials;
    if (ms) ms[c] = t_ms;
    if (bi < 0 || t_ms < best) {
      best = t_ms;
      bi = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) return s;
  B->grid = grids[(bi % 6) >> 1];
  B->dynamic = (bi & 1) == 0;
  B->layout = layouts[bi / 6];
  if (B->graph) {                     // the next step captures the tuned launches
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
  }
  if (grid) *grid = B->grid;
  if (dynamic) *dynamic = B->dynamic ? 1 : 0;
  if (layout) *layout = B->layout;
  return batch_status(B);
}

agile_status agile_batch_create(const agile_config* cfgs, int nsolve, const agile_allocator* alloc,
                                void* stream, agile_batch** out) {
  if (!cfgs || !out || nsolve < 1 || nsolve > (1 << 20)) return AGILE_EINVAL;
  *out = nullptr;
  const agile_config& c0 = cfgs[0];
  for (int i = 0; i < nsolve; ++i)
    if (!batch_cfg_ok(c0, cfgs[i])) return AGILE_EINVAL;
  agile_batch* B = new agile_batch();
  B->cfg = c0;
  B->nsolve = nsolve;
  B->cfgs.assign(cfgs, cfgs + nsolve);
  if (alloc && alloc->alloc && alloc->free) {
    B->alloc = *alloc;
    B->default_alloc = false;
  }
  B->stream = (cudaStream_t)stream;
  if (!B->stream) {   // graphs cannot be captured on the legacy default stream
    if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete B;
      return AGILE_ECUDA;
    }
    B->own_stream = true;
  }
  B->nv = cfg_nvar(c0);
  B->na = c0.physics == AGILE_SRHD ? 2 : 0;
  B->nt = B->nv + B->na;
  B->rb = c0.real_bytes;
  B->ics.assign(nsolve, nullptr);
  B->ic_users.assign(nsolve, nullptr);
  int nblk = 0;
  for (int i = 0; i < nsolve; ++i) {
    HostMesh* hm = new HostMesh(cfgs[i].base_blocks, cfgs[i].max_level, cfgs[i].bc, cfgs[i].xmin, cfgs[i].xmax);
    B->meshes.push_back(hm);
    B->offset.push_back(nblk);
    B->live.push_back(1);
    nblk += (int)hm->blocks().size();
  }
  B->cap = nblk;
  B->scap = nsolve;
  agile_mesh view;
  as_mesh_view(B, &view);
  view.nblk = nblk;
  const size_t pool = (size_t)nblk * B->nt * NCELL * B->rb;
  B->U[0] = dalloc(&view, pool);
  B->d_status = (int*)dalloc(&view, sizeof(int));
  B->d_speeds = (unsigned long long*)dalloc(&view, 2 * sizeof(unsigned long long) * nsolve);
  B->d_dtch = (double*)dalloc(&view, 2 * sizeof(double) * nsolve);
  B->d_work = (int*)dalloc(&view, 4 * sizeof(int));
  if (!B->U[0] || !B->d_status || !B->d_speeds || !B->d_dtch || !B->d_work) {
    agile_batch_destroy(B);
    return AGILE_ENOMEM;
  }
  if (cudaMemsetAsync(B->d_status, 0, sizeof(int), B->stream) != cudaSuccess ||
      cudaMemsetAsync(B->U[0], 0, pool, B->stream) != cudaSuccess) {
    agile_batch_destroy(B);
    return AGILE_ECUDA;
  }
  const agile_status st = batch_rebuild(B);
  if (st) {
    agile_batch_destroy(B);
    return st;
  }
  *out = B;
  return AGILE_OK;
}

void agile_batch_destroy(agile_batch* B) {
  if (!B) return;
  cudaStreamSynchronize(B->stream);
  if (B->graph) cudaGraphExecDestroy(B->graph);
  agile_mesh view;
  as_mesh_view(B, &view);
  for (int i = 0; i < 3; ++i) dfree(&view, B->U[i]);
  dfree_t(&view, B->d_bd);
  dfree_t(&view, B->d_solve_of);
  dfree_t(&view, B->d_status);
  dfree_t(&view, B->d_speeds);
  dfree_t(&view, B->d_dtch);
  dfree_t(&view, B->d_work);
  dfree_t(&view, B->d_wl);
  dfree_t(&view, B->d_ghosts);
  dfree_t(&view, B->d_fix);
  dfree(&view, B->G);
  dfree(&view, B->FR);
  dfree(&view, B->W);
  dfree(&view, B->WG);
  cudaStreamSynchronize(B->stream);
  batch_reap_uploads(B, true);
  if (B->up_stream) {
    cudaStreamSynchronize(B->up_stream);
    cudaStreamDestroy(B->up_stream);
  }
  for (HostMesh* hm : B->meshes) delete hm;   // nullptr for detached solves
  if (B->own_stream) cudaStreamDestroy(B->stream);
  delete B;
}

agile_status agile_batch_layout(agile_batch* B, int solve, size_t* nblocks, int* nvar) {
  if (!solve_ok(B, solve)) return AGILE_EINVAL;
  if (nblocks) *nblocks = B->meshes[solve]->blocks().size();
  if (nvar) *nvar = B->nv;
  return AGILE_OK;
}

agile_status agile_batch_set_state(agile_batch* B, int solve, agile_ic_fn ic, void* user) {
  if (!ic || !solve_ok(B, solve)) return bfail(B, AGILE_EINVAL, "bad argument");
  agile_mesh view;
  as_mesh_view(B, &view);
  view.mesh = B->meshes[solve];
  view.cfg = B->cfgs[solve];
  view.ic = ic;
  view.ic_user = user;
  view.d_status = B->d_status;
  std::vector<int> blocks(B->meshes[solve]->blocks().size());
  for (size_t i = 0; i < blocks.size(); ++i) blocks[i] = B->offset[solve] + (int)i;
  // apply_ic converts with the block's key from view.mesh: pass local indices through a
  // pool pointer shifted to this solve's first block
  std::vector<int> local(blocks.size());
  for (size_t i = 0; i < local.size(); ++i) local[i] = (int)i;
  char* base = (char*)B->U[0] + (size_t)B->offset[solve] * B->nt * NCELL * B->rb;
  view.nblk = (int)local.size();
  agile_status s = apply_ic(&view, base, local);
  view.mesh = nullptr;
  if (s) return bfail(B, s, view.err);
  B->ics[solve] = ic;
  B->ic_users[solve] = user;
  B->speeds_valid = false;
  return batch_status(B);
}

agile_status agile_batch_set_state_prims(agile_batch* B, int solve, const double* prim, size_t nblk) {
  if (!prim || !solve_ok(B, solve)) return bfail(B, AGILE_EINVAL, "bad argument");
  if (nblk != B->meshes[solve]->blocks().size()) return bfail(B, AGILE_EINVAL, "block count does not match the solve");
  agile_mesh view;
  as_mesh_view(B, &view);
  view.mesh = B->meshes[solve];
  view.cfg = B->cfgs[solve];
  view.ic = nullptr;
  view.ic_user = nullptr;
  view.d_status = B->d_status;
  // the primitives and the local block indices uploaded without waiting for the steps
  // already enqueued, converted on the batch stream after them
  std::vector<int> local(nblk);
  for (size_t i = 0; i < nblk; ++i) local[i] = (int)i;
  char* base = (char*)B->U[0] + (size_t)B->offset[solve] * B->nt * NCELL * B->rb;
  agile_status s = AGILE_OK;
  const size_t pbytes = nblk * B->nv * NCELL * sizeof(double), lbytes = nblk * sizeof(int);
  size_t pcap = 0, lcap = 0;
  void* d_prim = batch_upload(B, prim, pbytes, &s, &pcap);
  if (!d_prim) return s;
  void* d_local = batch_upload(B, local.data(), lbytes, &s, &lcap);
  if (!d_local) {
    batch_upload_done(B, d_prim, pcap);
    return s;
  }
  view.nblk = (int)nblk;
  AuxArgs a = aux_args(&view, base);
  const cudaError_t e = launch_prim2cons(a, (const double*)d_prim, (const int*)d_local, (int)nblk, B->stream);
  view.mesh = nullptr;
  s = batch_upload_done(B, d_prim, pcap);
  const agile_status s2 = batch_upload_done(B, d_local, lcap);
  if (e != cudaSuccess) return bfail(B, AGILE_ECUDA, std::string("prim2cons: ") + cudaGetErrorString(e));
  if (s) return s;
  if (s2) return s2;
  B->ics[solve] = nullptr;
  B->ic_users[solve] = nullptr;
  B->speeds_valid = false;
  return AGILE_OK;                            // enqueued; errors surface at the next sync
}

agile_status agile_batch_step(agile_batch* B) {
  if (!B) return AGILE_EINVAL;
  agile_status s = B->W ? AGILE_OK : batch_ensure_speeds(B);   // SRHD: the first pass reduces them
  if (s) return s;
  if (B->steps_done == 0) {   // first step eagerly: sets kernel attributes outside any capture
    s = batch_enqueue_step(B);
    if (s) return s;
  } else {
    if (!B->graph) {
      cudaGraph_t g = nullptr;
      BCK(B, cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
      s = batch_enqueue_step(B);
      cudaGraph_t gg = nullptr;
      cudaError_t e = cudaStreamEndCapture(B->stream, &gg);
      if (s) {
        if (gg) cudaGraphDestroy(gg);
        return s;
      }
      if (e != cudaSuccess) return bfail(B, AGILE_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      g = gg;
      e = cudaGraphInstantiate(&B->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return bfail(B, AGILE_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    BCK(B, cudaGraphLaunch(B->graph, B->stream));
  }
  B->launches += B->cfg.rk + 1 + (B->cfg.physics == AGILE_MHD_GLM ? 1 : 0) +
                 (B->nghost ? B->cfg.rk : 0) +
                 (B->nfix ? B->cfg.rk + (B->W ? 0 : 1) + (B->cfg.physics == AGILE_MHD_GLM ? 1 : 0) : 0) +
                 (B->W ? B->cfg.rk : 0);
  B->steps_done++;
  B->speeds_valid = B->W == nullptr;   // SRHD: U^{n+1}'s maxima come with the next step's first pass
  return AGILE_OK;
}

agile_status agile_batch_cfl_dt(agile_batch* B, double* dt) {
  if (!B || !dt) return bfail(B, AGILE_EINVAL, "null argument");
  agile_status s = batch_ensure_speeds(B);
  if (s) return s;
  std::vector<unsigned long long> h(2 * (size_t)B->nsolve);
  BCK(B, cudaMemcpyAsync(h.data(), B->d_speeds, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, B->stream));
  s = batch_status(B);
  if (s) return s;
  for (int i = 0; i < B->nsolve; ++i) {
    double smax;
    memcpy(&smax, &h[2 * i], sizeof(double));
    dt[i] = B->live[i] ? B->cfg.cfl / smax : 0.0;
  }
  return AGILE_OK;
}

agile_status agile_batch_get_state(agile_batch* B, int solve, int* level, int* ijk, double* cons) {
  if (!solve_ok(B, solve)) return bfail(B, AGILE_EINVAL, "bad argument");
  const auto& keys = B->meshes[solve]->blocks();
  const int n = (int)keys.size();
  for (int i = 0; i < n; ++i) {
    if (level) level[i] = keys[i].lev;
    if (ijk) {
      ijk[3 * i] = keys[i].x;
      ijk[3 * i + 1] = keys[i].y;
      ijk[3 * i + 2] = keys[i].z;
    }
  }
  if (!cons) return batch_status(B);
  agile_mesh view;
  as_mesh_view(B, &view);
  const size_t bytes = (size_t)n * B->nv * NCELL * sizeof(double);
  double* d = (double*)dalloc(&view, bytes);
  if (!d) return bfail(B, AGILE_ENOMEM, "device allocation failed");
  AuxArgs a = batch_aux(B, (char*)B->U[0] + (size_t)B->offset[solve] * B->nt * NCELL * B->rb);
  a.nblk = n;
  a.wl = nullptr;
  BCK(B, launch_pack(a, d, nullptr, B->stream));
  BCK(B, cudaMemcpyAsync(cons, d, bytes, cudaMemcpyDeviceToHost, B->stream));
  agile_status s = batch_status(B);
  dfree_t(&view, d);
  return s;
}

agile_status agile_batch_regrid_flags(agile_batch* B, int solve, const int* flags, int init, int* nr, int* nc) {
  if (!flags || !solve_ok(B, solve)) return bfail(B, AGILE_EINVAL, "bad argument");
  const int n = (int)B->meshes[solve]->blocks().size();
  std::vector<int> f(flags, flags + n);
  return batch_regrid(B, solve, f, init, nr, nc);
}

agile_status agile_batch_regrid(agile_batch* B, int solve, int init, int* nr, int* nc) {
  if (!B || solve < -1 || solve >= B->nsolve || (solve >= 0 && !B->live[solve]))
    return bfail(B, AGILE_EINVAL, "bad argument");
  std::vector<std::vector<int>> flags;
  agile_status s = batch_flags(B, &flags);
  if (s) return s;
  std::vector<RegridPlan> plans(B->nsolve);
  int tr = 0, tc = 0;
  for (int j = 0; j < B->nsolve; ++j) {
    if ((solve >= 0 && j != solve) || !B->live[j]) continue;
    plans[j] = B->meshes[j]->plan(flags[j]);
    tr += plans[j].n_refined;
    tc += plans[j].n_coarsened;
  }
  if (nr) *nr = tr;
  if (nc) *nc = tc;
  return batch_apply_plans(B, plans, init);
}

agile_status agile_batch_copy_solve(agile_batch* dst, int dst_solve, agile_batch* src, int src_solve) {
  if (!solve_ok(dst, dst_solve) || !solve_ok(src, src_solve)) return bfail(dst, AGILE_EINVAL, "bad argument");
  const agile_config& a = dst->cfgs[dst_solve];
  const agile_config& b = src->cfgs[src_solve];
  bool same = dst->nt == src->nt && dst->rb == src->rb && a.physics == b.physics && a.eos == b.eos;
  for (int d = 0; d < 3 && same; ++d)
    same = a.base_blocks[d] == b.base_blocks[d] && a.xmin[d] == b.xmin[d] && a.xmax[d] == b.xmax[d];
  for (int f = 0; f < 6 && same; ++f) same = a.bc[f] == b.bc[f];
  const auto& kd = dst->meshes[dst_solve]->blocks();
  const auto& ks = src->meshes[src_solve]->blocks();
  const size_t n = kd.size();
  if (same && n == ks.size())
    for (size_t i = 0; i < n && same; ++i)
      same = kd[i].lev == ks[i].lev && kd[i].x == ks[i].x && kd[i].y == ks[i].y && kd[i].z == ks[i].z;
  if (!same) return bfail(dst, AGILE_EINVAL, "solves differ in blocks, domain, boundaries or scheme");
  agile_status s = batch_status(src);     // the source's pending work is complete and error-free
  if (s) return bfail(dst, s, "source batch: " + src->err);
  const size_t per = (size_t)dst->nt * NCELL * dst->rb;
  BCK(dst, cudaMemcpyAsync((char*)dst->U[0] + dst->offset[dst_solve] * per,
                           (const char*)src->U[0] + src->offset[src_solve] * per, n * per,
                           cudaMemcpyDeviceToDevice, dst->stream));
  dst->speeds_valid = false;
  return batch_status(dst);
}

// A membership change of one solve that has no coarse-fine faces (no ghost slots, ghost tasks
// or flux-register fix-ups), with the pool and its block tables at capacity: only the solve's
// own range of the block tables and the work list change. The other solves' descriptors stay
// where they are on the device (their slot offsets do not move, the solve contributing none),
// so the cost is that of the one solve plus the work list, not of the whole batch. Returns
// false (nothing changed) where these conditions do not hold; the caller then rebuilds.
bool batch_patch(agile_batch* B, int solve, bool attach, agile_status* st) {
  *st = AGILE_OK;
  if (B->tab_cap != B->cap || B->cap_stage != B->cap || !B->d_bd || !B->d_solve_of || !B->d_wl) return false;
  if (solve < 0 || solve >= (int)B->tables.size()) return false;
  agile_batch::Tables& T = B->tables[solve];
  if (attach && !T.valid) {
    std::string err;
    T.desc.clear();
    T.ghosts.clear();
    T.fix.clear();
    B->meshes[solve]->build_descs(&T.desc, &T.ghosts, &T.fix, &T.nslots, &err);
    if (!err.empty()) return false;
    T.order = slab_order(*B->meshes[solve]);
    T.valid = true;
  }
  if (!T.valid || !T.ghosts.empty() || !T.fix.empty() || T.nslots) return false;
  const int O = B->offset[solve], n = (int)T.desc.size();
  if (O < 0 || O + n > B->cap) return false;
  std::vector<BlockDesc> d(T.desc);
  for (BlockDesc& bd : d) {
    for (int f = 0; f < 6; ++f) {
      if (bd.src[f] <= SRC_SLOT0 || bd.slot[f] >= 0) return false;   // a slot after all
      if (bd.src[f] >= 0) {
        if (bd.src[f] >= n) return false;
        bd.src[f] += O;
      }
      for (int k = 0; k < 4; ++k) {
        if (bd.nbr[f][k] >= n) return false;
        if (bd.nbr[f][k] >= 0) bd.nbr[f][k] += O;
      }
    }
  }
  if (!attach) {                    // the range becomes a hole: inert descriptors
    BlockDesc inert{};
    for (int f = 0; f < 6; ++f) {
      inert.src[f] = SRC_OUTFLOW;
      inert.slot[f] = -1;
      inert.kind[f] = FK_BC;
      for (int q = 0; q < 4; ++q) inert.nbr[f][q] = -1;
    }
    inert.dx[0] = inert.dx[1] = inert.dx[2] = 1.0;
    inert.level = 1;
    std::fill(d.begin(), d.end(), inert);
  }
  std::vector<int> so(n, attach ? solve : 0), work;
  work.reserve(B->nwork + (attach ? n : 0));
  int extent = 0;
  for (int i = 0; i < B->nsolve; ++i) {      // the work list: live solves in index order
    if (!B->live[i] || (!attach && i == solve)) continue;
    const int c = solve_blocks(B, i);
    const agile_batch::Tables& Ti = B->tables[i];
    if (!Ti.valid || (int)Ti.order.size() != c) return false;
    for (int q : Ti.order) work.push_back(B->offset[i] + q);
    extent = std::max(extent, B->offset[i] + c);
  }
  // one upload of [descriptors | solve indices | work list], copied into place on the batch
  // stream behind the steps that still read the old work list
  const size_t bd_bytes = d.size() * sizeof(BlockDesc), so_bytes = so.size() * sizeof(int);
  const size_t wl_bytes = work.size() * sizeof(int);
  std::vector<char> h(bd_bytes + so_bytes + wl_bytes + 1);
  memcpy(h.data(), d.data(), bd_bytes);
  memcpy(h.data() + bd_bytes, so.data(), so_bytes);
  memcpy(h.data() + bd_bytes + so_bytes, work.data(), wl_bytes);
  size_t dcap = 0;
  char* dev = (char*)batch_upload(B, h.data(), h.size(), st, &dcap);
  if (!dev) return true;
  auto cp = [&](void* dst, const char* src, size_t bytes) {
    if (!bytes || *st) return;
    const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, B->stream);
    if (e != cudaSuccess) *st = bfail(B, AGILE_ECUDA, std::string("table copy: ") + cudaGetErrorString(e));
  };
  cp(B->d_bd + O, dev, bd_bytes);
  cp(B->d_solve_of + O, dev + bd_bytes, so_bytes);
  cp(B->d_wl, dev + bd_bytes + so_bytes, wl_bytes);
  const agile_status sd = batch_upload_done(B, dev, dcap);
  if (!*st) *st = sd;
  if (*st) return true;
  B->nwork = (int)work.size();
  B->nblk = std::max(B->nblk, extent);       // per-block scratch covers every pool block in use
  if (!attach) T = agile_batch::Tables();
  if (B->graph) {                            // the captured step refers to the old work list
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
  }
  B->steps_done = 0;
  B->speeds_valid = false;
  return true;
}

// A new pool of ncap blocks with the live solves copied into it compactly, in index order;
// *end (may be NULL) receives the first free block. The caller rebuilds the tables (the
// stage buffers follow the capacity there).
agile_status batch_repool(agile_batch* B, int ncap, int* end) {
  agile_mesh view;
  as_mesh_view(B, &view);
  const size_t per = (size_t)B->nt * NCELL * B->rb;
  void* Unew = dalloc(&view, (size_t)std::max(ncap, 1) * per);
  if (!Unew) return bfail(B, AGILE_ENOMEM, "device allocation failed");
  std::vector<int> noff(B->nsolve, 0);
  int o = 0;
  for (int i = 0; i < B->nsolve; ++i) {
    if (!B->live[i]) continue;
    const int c = solve_blocks(B, i);
    if (o + c > ncap) {
      dfree(&view, Unew);
      return bfail(B, AGILE_EINVAL, "new pool smaller than the live solves");
    }
    if (c) {
      const cudaError_t e = cudaMemcpyAsync((char*)Unew + (size_t)o * per,
                                            (const char*)B->U[0] + (size_t)B->offset[i] * per, (size_t)c * per,
                                            cudaMemcpyDeviceToDevice, B->stream);
      if (e != cudaSuccess) {
        dfree(&view, Unew);
        return bfail(B, AGILE_ECUDA, std::string("pool copy: ") + cudaGetErrorString(e));
      }
    }
    noff[i] = o;
    o += c;
  }
  for (int i = 0; i < B->nsolve; ++i)
    if (B->live[i]) B->offset[i] = noff[i];
  dfree(&view, B->U[0]);                     // in stream order, after the copies
  B->U[0] = Unew;
  B->cap = ncap;
  if (end) *end = o;
  return AGILE_OK;
}

agile_status agile_batch_attach(agile_batch* B, const agile_config* cfg, int* solve) {
  if (!B || !cfg || !solve) return bfail(B, AGILE_EINVAL, "null argument");
  if (!batch_cfg_ok(B->cfg, *cfg)) return bfail(B, AGILE_EINVAL, "the solve's scheme differs from the batch's");
  agile_status s = AGILE_OK;
  std::unique_ptr<HostMesh> hm(new HostMesh(cfg->base_blocks, cfg->max_level, cfg->bc, cfg->xmin, cfg->xmax));
  const int n = (int)hm->blocks().size();
  int idx = -1;                              // a detached solve's index is reused
  for (int i = 0; i < B->nsolve && idx < 0; ++i)
    if (!B->live[i]) idx = i;
  if (idx < 0) {                             // per-solve device arrays first: nothing moved yet
    s = batch_reserve_solves(B, B->nsolve + 1);
    if (s) return s;
  }
  // first fit among the holes between live solves, else after the last one
  std::vector<std::pair<int, int>> ranges;   // (offset, count) of live solves, sorted
  for (int i = 0; i < B->nsolve; ++i)
    if (B->live[i]) ranges.push_back({B->offset[i], solve_blocks(B, i)});
  std::sort(ranges.begin(), ranges.end());
  int at = -1, prev = 0;
  for (const auto& r : ranges) {
    if (r.first - prev >= n) {
      at = prev;
      break;
    }
    prev = r.first + r.second;
  }
  if (at < 0 && B->cap - prev >= n) at = prev;
  agile_mesh view;
  as_mesh_view(B, &view);
  const size_t per = (size_t)B->nt * NCELL * B->rb;
  if (at < 0) {
    // grow: a new pool with room for this solve and a quarter more, the live solves copied
    // into it compactly
    int live_blocks = 0;
    for (const auto& r : ranges) live_blocks += r.second;
    s = batch_repool(B, live_blocks + n + std::max(n, (live_blocks + n) / 4), &at);
    if (s) return s;
  }
  if (idx < 0) {
    idx = B->nsolve++;
    B->cfgs.push_back(*cfg);
    B->meshes.push_back(nullptr);
    B->offset.push_back(0);
    B->live.push_back(0);
    B->ics.push_back(nullptr);
    B->ic_users.push_back(nullptr);
  }
  B->cfgs[idx] = *cfg;
  B->meshes[idx] = hm.release();
  B->offset[idx] = at;
  B->live[idx] = 1;
  B->tables.resize(B->nsolve);
  B->tables[idx].valid = false;
  B->ics[idx] = nullptr;
  B->ic_users[idx] = nullptr;
  BCK(B, cudaMemsetAsync((char*)B->U[0] + (size_t)at * per, 0, (size_t)n * per, B->stream));
  if (!batch_patch(B, idx, true, &s)) s = batch_rebuild(B);
  if (s) return s;
  *solve = idx;
  return AGILE_OK;
}

agile_status agile_batch_detach(agile_batch* B, int solve) {
  if (!solve_ok(B, solve)) return bfail(B, AGILE_EINVAL, "bad argument");
  agile_status s = AGILE_OK;
  const bool patched = batch_patch(B, solve, false, &s);   // reads the solve's tables and mesh
  delete B->meshes[solve];
  B->meshes[solve] = nullptr;
  B->live[solve] = 0;
  B->ics[solve] = nullptr;
  B->ic_users[solve] = nullptr;
  if (s) return s;
  // a pool less than 60% used shrinks to its live blocks and a quarter more, so that the
  // capacity follows the attached solves down as well as up (at most 1/0.6 times them)
  int live_blocks = 0;
  for (int i = 0; i < B->nsolve; ++i) live_blocks += solve_blocks(B, i);
  if (B->cap > 4096 && 5LL * live_blocks < 3LL * B->cap) {
    s = batch_repool(B, live_blocks + live_blocks / 4, nullptr);
    if (s) return s;
    return batch_rebuild(B);
  }
  return patched ? AGILE_OK : batch_rebuild(B);
}

agile_status agile_batch_sync(agile_batch* B) {
  if (!B) return AGILE_EINVAL;
  return batch_status(B);
}

long long agile_batch_launches(const agile_batch* B) { return B ? B->launches : 0; }

const char* agile_batch_last_error(const agile_batch* B) { return B ? B->err.c_str() : "null batch"; }

}  // extern "C"
