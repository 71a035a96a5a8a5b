// Host octree of 16^3 blocks: neighbour classification (srl / c / f), 2:1-balanced
// refine/coarsen planning and the device descriptor tables (the paper's nbinfo lists,
// Section 2.1.3, rebuilt on every grid change).
#include "mesh.h"

#include <algorithm>
#include <deque>

namespace agile {

uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  uint64_t m = 0;
  for (int b = 0; b < 21; ++b) {
    m |= (uint64_t)((x >> b) & 1u) << (3 * b);
    m |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
    m |= (uint64_t)((z >> b) & 1u) << (3 * b + 2);
  }
  return m;
}

static bool key_less(const Key& a, const Key& b) {
  if (a.lev != b.lev) return a.lev < b.lev;
  return morton3(a.x, a.y, a.z) < morton3(b.x, b.y, b.z);
}

HostMesh::HostMesh(const int base[3], int max_level, const int bc[6], const double xmin[3],
                   const double xmax[3]) {
  for (int d = 0; d < 3; ++d) {
    base_[d] = base[d];
    xmin_[d] = xmin[d];
    xmax_[d] = xmax[d];
    periodic_[d] = bc[2 * d] == BC_PERIODIC;
  }
  for (int f = 0; f < 6; ++f) bc_[f] = bc[f];
  max_level_ = max_level;
  for (int z = 0; z < base[2]; ++z)
    for (int y = 0; y < base[1]; ++y)
      for (int x = 0; x < base[0]; ++x) blocks_.push_back(Key{1, x, y, z});
  reindex();
}

void HostMesh::reindex() {
  std::sort(blocks_.begin(), blocks_.end(), key_less);
  index_.clear();
  index_.reserve(blocks_.size() * 2);
  for (size_t i = 0; i < blocks_.size(); ++i) index_[key_code(blocks_[i])] = (int)i;
}

int HostMesh::find(const Key& k) const {
  auto it = index_.find(key_code(k));
  return it == index_.end() ? -1 : it->second;
}

double HostMesh::dx(int lev, int d) const {
  return (xmax_[d] - xmin_[d]) / ((double)base_[d] * NB * (double)(1 << (lev - 1)));
}

bool HostMesh::neighbour_pos(const Key& k, int ox, int oy, int oz, Key* out) const {
  int p[3] = {k.x + ox, k.y + oy, k.z + oz};
  for (int d = 0; d < 3; ++d) {
    const int n = nblocks_dim(k.lev, d);
    if (p[d] < 0 || p[d] >= n) {
      if (!periodic_[d]) return false;
      p[d] = ((p[d] % n) + n) % n;
    }
  }
  *out = Key{k.lev, p[0], p[1], p[2]};
  return true;
}

int HostMesh::covering_leaf(const Key& k) const {
  Key q = k;
  while (q.lev >= 1) {
    const int i = find(q);
    if (i >= 0) return i;
    q = Key{q.lev - 1, q.x >> 1, q.y >> 1, q.z >> 1};
  }
  return -1;
}

FaceInfo HostMesh::face(int i, int f) const {
  FaceInfo fi;
  fi.kind = FK_BC;
  fi.bc = bc_[f];
  fi.nbr[0] = fi.nbr[1] = fi.nbr[2] = fi.nbr[3] = -1;
  fi.par[0] = fi.par[1] = fi.par[2] = 0;
  const Key& k = blocks_[i];
  const int d = f >> 1;
  const int s = (f & 1) ? 1 : -1;
  int o[3] = {0, 0, 0};
  o[d] = s;
  Key n;
  if (!neighbour_pos(k, o[0], o[1], o[2], &n)) return fi;
  int j = find(n);
  if (j >= 0) {
    fi.kind = FK_SAME;
    fi.nbr[0] = j;
    return fi;
  }
  if (k.lev > 1) {
    j = find(Key{k.lev - 1, n.x >> 1, n.y >> 1, n.z >> 1});
    if (j >= 0) {
      fi.kind = FK_COARSER;
      fi.nbr[0] = j;
      fi.par[0] = n.x & 1;
      fi.par[1] = n.y & 1;
      fi.par[2] = n.z & 1;
      return fi;
    }
  }
  fi.kind = FK_FINER;
  const int t1d = d == 0 ? 1 : 0;
  const int t2d = d == 2 ? 1 : 2;
  const int np[3] = {n.x, n.y, n.z};
  for (int t2 = 0; t2 < 2; ++t2)
    for (int t1 = 0; t1 < 2; ++t1) {
      int c[3];
      c[d] = 2 * np[d] + (s < 0 ? 1 : 0);
      c[t1d] = 2 * np[t1d] + t1;
      c[t2d] = 2 * np[t2d] + t2;
      fi.nbr[t1 + 2 * t2] = find(Key{k.lev + 1, c[0], c[1], c[2]});
    }
  return fi;
}

RegridPlan HostMesh::plan(const std::vector<int>& flags) const {
  RegridPlan P;
  const int n = (int)blocks_.size();
  std::vector<char> refine(n, 0);
  std::deque<int> work;
  for (int i = 0; i < n; ++i)
    if (flags[i] > 0 && blocks_[i].lev < max_level_) {
      refine[i] = 1;
      work.push_back(i);
    }
  // 2:1 closure: a refined leaf forces its coarser face/edge/corner neighbours to refine.
  while (!work.empty()) {
    const int i = work.front();
    work.pop_front();
    const Key& k = blocks_[i];
    for (int oz = -1; oz <= 1; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          if (!ox && !oy && !oz) continue;
          Key q;
          if (!neighbour_pos(k, ox, oy, oz, &q)) continue;
          const int j = covering_leaf(q);
          if (j >= 0 && blocks_[j].lev < k.lev && !refine[j]) {
            refine[j] = 1;
            work.push_back(j);
          }
        }
  }
  // Nodes with children after refinement.
  std::unordered_set<uint64_t> internal;
  for (int i = 0; i < n; ++i) {
    Key q = blocks_[i];
    while (q.lev > 1) {
      q = Key{q.lev - 1, q.x >> 1, q.y >> 1, q.z >> 1};
      if (!internal.insert(key_code(q)).second) break;
    }
    if (refine[i]) internal.insert(key_code(blocks_[i]));
  }
  // Coarsening candidates: parents whose 8 children are leaves flagged -1, none refined,
  // and no block adjacent to the parent refined in the post-refinement tree.
  std::vector<char> coarsen(n, 0);
  std::vector<Key> new_parents;
  std::vector<std::vector<int>> parent_kids;
  std::unordered_set<uint64_t> seen;
  for (int i = 0; i < n; ++i) {
    const Key& k = blocks_[i];
    if (k.lev < 2) continue;
    const Key pk{k.lev - 1, k.x >> 1, k.y >> 1, k.z >> 1};
    if (!seen.insert(key_code(pk)).second) continue;
    std::vector<int> kids(8, -1);
    bool ok = true;
    for (int o = 0; o < 8 && ok; ++o) {
      const int j = find(Key{k.lev, 2 * pk.x + (o & 1), 2 * pk.y + ((o >> 1) & 1),
                             2 * pk.z + (o >> 2)});
      if (j < 0 || flags[j] != -1 || refine[j]) ok = false;
      kids[o] = j;
    }
    if (!ok) continue;
    for (int o = 0; o < 8 && ok; ++o) {
      const Key& c = blocks_[kids[o]];
      for (int oz = -1; oz <= 1 && ok; ++oz)
        for (int oy = -1; oy <= 1 && ok; ++oy)
          for (int ox = -1; ox <= 1 && ok; ++ox) {
            if (!ox && !oy && !oz) continue;
            Key q;
            if (!neighbour_pos(c, ox, oy, oz, &q)) continue;
            if ((q.x >> 1) == pk.x && (q.y >> 1) == pk.y && (q.z >> 1) == pk.z) continue;
            if (internal.count(key_code(q))) ok = false;
          }
    }
    if (!ok) continue;
    for (int o = 0; o < 8; ++o) coarsen[kids[o]] = 1;
    new_parents.push_back(pk);
    parent_kids.push_back(kids);
  }
  // New leaf list with its sources.
  struct Item {
    Key k;
    RegridSrc s;
    bool created;
  };
  std::vector<Item> items;
  for (int i = 0; i < n; ++i) {
    const Key& k = blocks_[i];
    if (refine[i]) {
      ++P.n_refined;
      for (int o = 0; o < 8; ++o) {
        Item it;
        it.k = Key{k.lev + 1, 2 * k.x + (o & 1), 2 * k.y + ((o >> 1) & 1), 2 * k.z + (o >> 2)};
        it.s.mode = 1;
        it.s.octant = o;
        for (int q = 0; q < 8; ++q) it.s.src[q] = q == 0 ? i : -1;
        it.created = true;
        items.push_back(it);
      }
    } else if (!coarsen[i]) {
      Item it;
      it.k = k;
      it.s.mode = 0;
      it.s.octant = 0;
      for (int q = 0; q < 8; ++q) it.s.src[q] = q == 0 ? i : -1;
      it.created = false;
      items.push_back(it);
    }
  }
  for (size_t p = 0; p < new_parents.size(); ++p) {
    Item it;
    it.k = new_parents[p];
    it.s.mode = 2;
    it.s.octant = 0;
    for (int q = 0; q < 8; ++q) it.s.src[q] = parent_kids[p][q];
    it.created = true;
    items.push_back(it);
  }
  P.n_coarsened = (int)new_parents.size();
  std::sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return key_less(a.k, b.k); });
  for (size_t i = 0; i < items.size(); ++i) {
    P.blocks.push_back(items[i].k);
    P.src.push_back(items[i].s);
    if (items[i].created) P.created.push_back((int)i);
  }
  return P;
}

void HostMesh::apply(const RegridPlan& p) {
  blocks_ = p.blocks;
  reindex();
}

void HostMesh::build_descs(std::vector<BlockDesc>* desc, std::vector<GhostTask>* ghosts,
                           std::vector<FixupTask>* fixups, int* nslots, std::string* err) const {
  const int n = (int)blocks_.size();
  desc->assign(n, BlockDesc{});
  ghosts->clear();
  fixups->clear();
  int ns = 0;
  std::vector<FaceInfo> fis((size_t)n * 6);
  for (int i = 0; i < n; ++i) {
    BlockDesc& bd = (*desc)[i];
    const Key& k = blocks_[i];
    bd.level = k.lev;
    for (int d = 0; d < 3; ++d) bd.dx[d] = dx(k.lev, d);
    for (int f = 0; f < 6; ++f) {
      const FaceInfo fi = face(i, f);
      fis[(size_t)i * 6 + f] = fi;
      bd.kind[f] = fi.kind;
      bd.slot[f] = -1;
      for (int q = 0; q < 4; ++q) bd.nbr[f][q] = fi.nbr[q];
      if (fi.kind == FK_SAME) {
        bd.src[f] = fi.nbr[0];
      } else if (fi.kind == FK_BC) {
        if (fi.bc == BC_OUTFLOW) bd.src[f] = SRC_OUTFLOW;
        else if (fi.bc == BC_REFLECT) bd.src[f] = SRC_REFLECT;
        else { if (err) *err = "periodic face without neighbour"; return; }
      } else {
        if (fi.kind == FK_FINER)
          for (int q = 0; q < 4; ++q)
            if (fi.nbr[q] < 0) { if (err) *err = "mesh is not 2:1 balanced"; return; }
        bd.slot[f] = ns;
        bd.src[f] = SRC_SLOT0 - ns;
        GhostTask g;
        g.blk = i;
        g.face = f;
        g.kind = fi.kind;
        g.slot = ns;
        for (int q = 0; q < 4; ++q) g.nbr[q] = fi.nbr[q];
        for (int q = 0; q < 3; ++q) g.par[q] = fi.par[q];
        g.pad = 0;
        ghosts->push_back(g);
        ++ns;
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    const BlockDesc& bd = (*desc)[i];
    FixupTask t;
    t.blk = i;
    t.nface = 0;
    for (int f = 0; f < 6; ++f) {
      if (bd.kind[f] != FK_FINER) continue;
      const int j = t.nface++;
      t.face[j] = f;
      t.slot_c[j] = bd.slot[f];
      for (int q = 0; q < 4; ++q) {
        const int fb = bd.nbr[f][q];
        t.slot_f[j][q] = (*desc)[fb].slot[f ^ 1];
        if (t.slot_f[j][q] < 0 || (*desc)[fb].kind[f ^ 1] != FK_COARSER) {
          if (err) *err = "inconsistent coarse-fine face";
          return;
        }
      }
    }
    if (t.nface) fixups->push_back(t);
  }
  *nslots = ns;
}

bool HostMesh::balanced() const {
  for (size_t i = 0; i < blocks_.size(); ++i) {
    const Key& k = blocks_[i];
    for (int oz = -1; oz <= 1; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          if (!ox && !oy && !oz) continue;
          Key q;
          if (!neighbour_pos(k, ox, oy, oz, &q)) continue;
          const int j = covering_leaf(q);
          if (j >= 0) {
            if (k.lev - blocks_[j].lev > 1) return false;
          } else {
            // refined: the children touching k must be leaves
            const int o[3] = {ox, oy, oz};
            const int qp[3] = {q.x, q.y, q.z};
            for (int c = 0; c < 8; ++c) {
              int cp[3];
              bool touch = true;
              for (int d = 0; d < 3; ++d) {
                const int bit = (c >> d) & 1;
                if (o[d] > 0 && bit != 0) touch = false;
                if (o[d] < 0 && bit != 1) touch = false;
                cp[d] = 2 * qp[d] + bit;
              }
              if (touch && find(Key{k.lev + 1, cp[0], cp[1], cp[2]}) < 0) return false;
            }
          }
        }
  }
  return true;
}

}  // namespace agile
