// Host book-keeping of the block octree (paper Section 2.1.2 and Figs. 1-2: the grid,
// its connectivity and the refine/coarsen decisions live on the host; data stays on the
// device). Leaves are kept sorted by level, then Morton index.
#pragma once
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "agile_internal.h"

namespace agile {

struct Key {
  int lev, x, y, z;
};

inline uint64_t key_code(const Key& k) {
  return ((uint64_t)k.lev << 57) | ((uint64_t)(uint32_t)k.x << 38) |
         ((uint64_t)(uint32_t)k.y << 19) | (uint64_t)(uint32_t)k.z;
}

uint64_t morton3(uint32_t x, uint32_t y, uint32_t z);

struct FaceInfo {
  int kind;      // FK_*
  int bc;        // BC_* for FK_BC
  int nbr[4];    // same: [0]; coarser: [0]; finer: t1 + 2 t2
  int par[3];    // coarser: neighbour block position parity
};

struct RegridPlan {
  std::vector<Key> blocks;         // new leaves in order
  std::vector<RegridSrc> src;      // per new leaf
  std::vector<int> created;        // indices (new order) of refined children / new parents
  int n_refined = 0;
  int n_coarsened = 0;
};

class HostMesh {
 public:
  HostMesh(const int base[3], int max_level, const int bc[6], const double xmin[3],
           const double xmax[3]);

  const std::vector<Key>& blocks() const { return blocks_; }
  int find(const Key& k) const;
  bool has(const Key& k) const { return find(k) >= 0; }
  int nblocks_dim(int lev, int d) const { return base_[d] << (lev - 1); }
  double dx(int lev, int d) const;
  // Block position moved by (dx, dy, dz) at its level, wrapped on periodic axes;
  // false when it leaves the domain.
  bool neighbour_pos(const Key& k, int ox, int oy, int oz, Key* out) const;
  FaceInfo face(int i, int f) const;
  // Leaf covering block position k (level k.lev or coarser), -1 if k is refined.
  int covering_leaf(const Key& k) const;

  RegridPlan plan(const std::vector<int>& flags) const;   // flags per leaf: +1/-1/0
  void apply(const RegridPlan& p);

  // Device descriptors for the current mesh.
  void build_descs(std::vector<BlockDesc>* desc, std::vector<GhostTask>* ghosts,
                   std::vector<FixupTask>* fixups, int* nslots, std::string* err) const;

  bool balanced() const;

 private:
  void reindex();
  int base_[3];
  int max_level_;
  int bc_[6];
  bool periodic_[3];
  double xmin_[3], xmax_[3];
  std::vector<Key> blocks_;
  std::unordered_map<uint64_t, int> index_;
};

}  // namespace agile
