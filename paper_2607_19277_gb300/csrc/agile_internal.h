// Internal data structures of the block-AMR library (host and device).
//
// Layout in HBM (structure of arrays, 16^3 interiors only):
//   state pool   U[block][var][z][y][x]        var = conserved (NV) then auxiliary (NA)
//   ghost slots  G[slot][var][layer][t2][t1]   2 x 16 x 16 face ghosts for faces whose
//                                              neighbour is coarser or finer
//   flux regs    F[slot][var][t2][t1]          the block's own boundary-face flux there
// Same-level halos are never stored: kernels read them from the neighbour's interior
// through BlockDesc::src, physical boundaries are computed on the fly, and only
// coarse-fine faces go through ghost slots (the paper's srl / f / c neighbour classes).
// Tangential coordinates of face d: d = x -> (t1, t2) = (y, z); y -> (x, z); z -> (x, y).
#pragma once
#include <stddef.h>
#include <stdint.h>

namespace agile {

constexpr int NB = 16;            // interior cells per block edge
constexpr int NCELL = NB * NB * NB;
constexpr int NFACE = 6;          // faces: -x, +x, -y, +y, -z, +z

enum FaceKind : int { FK_SAME = 0, FK_BC = 1, FK_COARSER = 2, FK_FINER = 3 };
enum BcKind : int { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECT = 2 };
enum PhysKind : int { PH_HD = 0, PH_MHD = 1, PH_SRHD = 2, PH_SRHD_SYNGE = 3, PH_FFHD = 4, PH_FFHD_HTC = 5 };

// src encoding: >= 0 same-level neighbour block; SRC_OUTFLOW / SRC_REFLECT physical
// boundary; <= SRC_SLOT0 ghost slot (SRC_SLOT0 - slot).
constexpr int SRC_OUTFLOW = -1;
constexpr int SRC_REFLECT = -2;
constexpr int SRC_SLOT0 = -3;

struct BlockDesc {
  int src[NFACE];
  int slot[NFACE];      // ghost slot / flux register of the face, -1 if none
  int kind[NFACE];
  int nbr[NFACE][4];    // finer: the 4 fine blocks (t1 + 2 t2); coarser: [0] = coarse block
  double dx[3];
  int level;
  int pad;
};

struct GhostTask {      // one coarse-fine face of a block, filled before each stage
  int blk;
  int face;
  int kind;             // FK_COARSER (prolong) or FK_FINER (restrict)
  int slot;
  int nbr[4];
  int par[3];           // neighbour position parity (coarser case): coarse offset 8 * par
  int pad;
};

struct FixupTask {      // all faces of one coarse block shared with 4 finer blocks each
  int blk;
  int nface;
  int face[NFACE];
  int slot_c[NFACE];
  int slot_f[NFACE][4];
};

struct RegridSrc {      // how a block of the new mesh is made from the old one
  int mode;             // 0 copy, 1 prolong (from parent), 2 restrict (from 8 children)
  int octant;           // prolong: child octant ox + 2 oy + 4 oz
  int src[8];           // old block indices
};

inline int face_dim(int f) { return f >> 1; }
inline int face_side(int f) { return (f & 1) ? 1 : -1; }

}  // namespace agile
