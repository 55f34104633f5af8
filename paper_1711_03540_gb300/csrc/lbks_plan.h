// Host-side planning of the register-resident kernel: how lattices become pieces
// (whole rings, haloed halves for cluster pairs, haloed segments), and how pieces are
// packed into work groups (bundles) of one block or a two-block cluster.  Plain C++
// (no device code), so that host tests can check it directly.
#pragma once

#include <algorithm>
#include <cstdint>
#include <initializer_list>
#include <utility>
#include <vector>

#include "lbks_internal.h"

namespace lbks {
namespace plan {

// Sites per tile of the plain kernel family (one thread per site, one block per tile).
constexpr int kPlainTileMax = 256;
constexpr int kPlainTileMin = 32;

// Sites per plain-family tile: the largest of 256, 128, 64 and 32 that still gives every
// SM two tiles, else 32.  A small workload (one lattice of a few thousand sites) in
// 256-site tiles runs on a few SMs, each doing 256 sites' FP64 arithmetic per step at
// GB300's low FP64 rate, while the rest idle; smaller tiles spread the same per-site
// work over more SMs.  Results do not depend on the tiling (each thread updates one
// site on its own).  Reservoir lattices' tiles also cover their 2 c_max ghost nodes.
inline int plain_tile_sites(const std::vector<int64_t>& Ns, bool reservoir, int cmax, int sms) {
  for (int t = kPlainTileMax; t > kPlainTileMin; t /= 2) {
    int64_t tiles = 0;
    for (int64_t n : Ns) tiles += (n + (reservoir ? 2 * cmax : 0) + t - 1) / t;
    if (tiles >= 2 * (int64_t)sms) return t;
  }
  return kPlainTileMin;
}

// The plain family's tiles: run by run, consecutive stretches of plain_tile_sites sites
// (the last one of a run shorter) covering [0, N) of each run, or [-c_max, N + c_max)
// for reservoir lattices; *tile receives the tile length (the launches' block size).
inline std::vector<Tile> plain_tiles(const std::vector<int64_t>& Ns, bool reservoir, int cmax, int sms, int* tile) {
  const int t = plain_tile_sites(Ns, reservoir, cmax, sms);
  std::vector<Tile> pt;
  for (int32_t r = 0; r < (int32_t)Ns.size(); ++r) {
    const int64_t g0 = reservoir ? -cmax : 0, g1 = reservoir ? Ns[r] + cmax : Ns[r];
    for (int64_t x = g0; x < g1; x += t) pt.push_back(Tile{r, (int32_t)x, (int32_t)std::min<int64_t>(t, g1 - x), 0});
  }
  *tile = t;
  return pt;
}

// One half of a ring of N sites for a cluster pair: own sites [x_own, x_own + len) of
// the ring with `halo` sites on each side, lengthened on the right until it splits
// into runs of S and S-1 sites; false if that takes more than NT threads.
inline bool plan_half(int32_t r, int64_t N, int64_t x_own, int64_t len, int halo, int S, int NT, Piece* p) {
  int64_t n = len + 2 * halo;
  int64_t V = (n + S - 1) / S;
  while (n <= V * (S - 1)) { ++n; V = (n + S - 1) / S; }
  if (V > NT) return false;
  *p = Piece{};
  p->run = r; p->t0 = 0; p->nthr = (int)V; p->n = (int)n;
  p->x0 = ((x_own - halo) % N + N) % N;
  p->st_lo = halo; p->st_hi = (int)(halo + len);
  p->halo = halo;
  return true;
}

// Pieces of every run for (S, NT): rings (whole lattices held by at most ring_cap
// threads: NT, or 2 NT for two-block clusters) and segments (for longer lattices,
// held by one block each, with c_max * kseg halo sites per side); false if some
// run cannot be held.  With two-block clusters and kx > 0, a lattice longer than one
// block holds is split into two halves (consecutive in `rings`, halo c_max kx) when
// each half with its halos fits one block, instead of one ring across both blocks.
inline bool plan_pieces(const std::vector<int64_t>& Ns, int C, int S, int NT, int ring_cap, int kseg, int kx,
                        std::vector<Piece>* rings, std::vector<Piece>* segs) {
  rings->clear();
  segs->clear();
  rings->reserve(Ns.size() + Ns.size() / 2);
  for (int32_t r = 0; r < (int32_t)Ns.size(); ++r) {
    const int64_t N = Ns[r];
    // Ring: hold m copies of the lattice around one ring of m N sites (m > 1 only
    // for lattices shorter than S (S-1), which cannot be cut into runs of S and
    // S-1 sites).  Translation invariance keeps the copies bitwise identical;
    // the first one is stored.
    bool ring = false;
    for (int64_t m = 1;; ++m) {
      const int64_t n = m * N;
      const int64_t V = (n + S - 1) / S;
      if (V > ring_cap) break;
      if (n > V * (S - 1)) {
        if (V > NT && kx > 0) {
          const int halo = C * kx;
          const int64_t NA = (N + 1) / 2, NB = N - NA;
          Piece a{}, b{};
          if (NB >= 2 * halo && plan_half(r, N, 0, NA, halo, S, NT, &a) && plan_half(r, N, NA, NB, halo, S, NT, &b)) {
            rings->push_back(a);
            rings->push_back(b);
            ring = true;
            break;
          }
        }
        Piece p{};
        p.run = r; p.t0 = 0; p.nthr = (int)V; p.n = (int)n; p.x0 = 0; p.st_lo = 0; p.st_hi = (int)N;
        rings->push_back(p);
        ring = true;
        break;
      }
    }
    if (ring) continue;
    const int64_t h2 = 2LL * C * kseg;
    const int64_t room = (int64_t)NT * S - h2 - 2 * S;
    if (room <= 0) return false;
    const int64_t nseg = (N + room - 1) / room;
    const int64_t Ls = (N + nseg - 1) / nseg;
    for (int64_t s0 = 0; s0 < N; s0 += Ls) {
      const int64_t len = std::min<int64_t>(Ls, N - s0);
      int64_t n = len + h2;
      int64_t V = (n + S - 1) / S;
      while (n <= V * (S - 1)) { ++n; V = (n + S - 1) / S; }
      if (V > NT) return false;
      Piece p{};
      p.run = r; p.t0 = 0; p.nthr = (int)V; p.n = (int)n;
      p.x0 = ((s0 - (int64_t)C * kseg) % N + N) % N;
      p.st_lo = C * kseg; p.st_hi = (int)(C * kseg + len);
      segs->push_back(p);
    }
  }
  return true;
}

// Indices 0..n-1 in decreasing order of k (k >= 0), equal keys in index order: the
// order of a stable sort, by counting (keys are thread counts, at most a few thousand).
inline std::vector<int> stable_desc(const std::vector<int>& k) {
  int kmax = 0;
  for (int v : k) kmax = std::max(kmax, v);
  std::vector<int> start((size_t)kmax + 2, 0);  // start[kmax - v]: first slot of key v
  for (int v : k) ++start[(size_t)(kmax - v) + 1];
  for (size_t q = 1; q < start.size(); ++q) start[q] += start[q - 1];
  std::vector<int> idx(k.size());
  for (size_t i = 0; i < k.size(); ++i) idx[(size_t)start[(size_t)(kmax - k[i])]++] = (int)i;
  return idx;
}

// Work groups of one lane during packing: first fit of pieces (threads nthr) into
// groups of `cap` threads.
struct Bins {
  int cap = 0;
  bool pair = false;  // pair work groups: block 0 is threads [0, cap/2), block 1 the rest
  // Members of each group in the order they joined it: a singly linked list over piece
  // indices (head, tail per group; nxt per piece), so that packing allocates nothing
  // per group.
  std::vector<int> head, tail, count, nxt;
  std::vector<int> used;   // threads [0, used) taken (pair work groups: the end of block 1's)
  std::vector<int> used0;  // pair work groups: threads [0, used0) of block 0 taken
  std::vector<int> key;    // queue order (largest first); empty: by occupied threads
  // Segment tree of the largest free run (block 0's or block 1's) over the groups, so
  // that first fit finds the first group with room in O(log groups).
  std::vector<int> tree;
  size_t tn = 0;

  size_t groups() const { return used.size(); }
  std::vector<int> members(size_t b) const {
    std::vector<int> m;
    for (int i = head[b]; i >= 0; i = nxt[(size_t)i]) m.push_back(i);
    return m;
  }
  void link(size_t b, int i) {
    if ((size_t)i >= nxt.size()) nxt.resize(std::max<size_t>((size_t)i + 1, 2 * nxt.size()), -1);
    nxt[(size_t)i] = -1;
    if (tail[b] < 0) head[b] = i;
    else nxt[(size_t)tail[b]] = i;
    tail[b] = i;
    ++count[b];
  }
  // A new, empty group with u0 threads of block 0 (pair groups) and threads [0, u)
  // (pair groups: block 1's up to u) taken.
  size_t new_group(int u0, int u) {
    head.push_back(-1);
    tail.push_back(-1);
    count.push_back(0);
    used.push_back(u);
    if (pair) used0.push_back(u0);
    return used.size() - 1;
  }
  int room(size_t b) const {
    int f = cap - used[b];
    if (pair) f = std::max(f, cap / 2 - used0[b]);
    return f;
  }
  void fix(size_t b) {
    if (b >= tn) {
      tn = std::max<size_t>(64, 2 * tn);
      while (tn <= b) tn *= 2;
      tree.assign(2 * tn, -1);
      for (size_t q = 0; q < used.size(); ++q) tree[tn + q] = room(q);
      for (size_t p = tn - 1; p >= 1; --p) tree[p] = std::max(tree[2 * p], tree[2 * p + 1]);
      return;
    }
    size_t p = tn + b;
    tree[p] = room(b);
    for (p >>= 1; p >= 1; p >>= 1) tree[p] = std::max(tree[2 * p], tree[2 * p + 1]);
  }
  // A new group holding pieces `mem`, with u0 and u as for new_group.
  void add(std::initializer_list<int> mem, int u0, int u) {
    const size_t b = new_group(u0, u);
    for (int i : mem) link(b, i);
    fix(b);
  }
  // First fit: the first group with room for the piece.  A piece never spans the
  // block edge of a pair work group here: it goes into block 0's free threads or
  // after block 1's taken ones.
  bool first_fit(std::vector<Piece>& pieces, int i) {
    const int need = pieces[i].nthr;
    if (tn == 0 || tree[1] < need) return false;
    size_t p = 1;
    while (p < tn) p = tree[2 * p] >= need ? 2 * p : 2 * p + 1;
    const size_t b = p - tn;
    if (pair && used0[b] + need <= cap / 2) {
      pieces[i].t0 = used0[b];
      used0[b] += need;
    } else {
      pieces[i].t0 = used[b];
      used[b] += need;
    }
    link(b, i);
    fix(b);
    return true;
  }
  void open(std::vector<Piece>& pieces, int i) {
    pieces[i].t0 = 0;
    add({i}, 0, pieces[i].nthr);
  }
  // bundles in decreasing order of occupied threads (longest first)
  void emit(const std::vector<Piece>& pieces, std::vector<Piece>* ordered, std::vector<int2>* bundles) const {
    const std::vector<int> order = stable_desc(key.empty() ? used : key);
    ordered->clear();
    bundles->clear();
    ordered->reserve(pieces.size());
    bundles->reserve(order.size());
    for (int b : order) {
      bundles->push_back(int2{(int)ordered->size(), count[(size_t)b]});
      for (int i = head[(size_t)b]; i >= 0; i = nxt[(size_t)i]) ordered->push_back(pieces[(size_t)i]);
    }
  }
};

inline std::vector<int> by_threads_desc(const std::vector<Piece>& pieces) {
  std::vector<int> nthr(pieces.size());
  for (size_t i = 0; i < pieces.size(); ++i) nthr[i] = pieces[i].nthr;
  return stable_desc(nthr);
}

// First-fit decreasing packing of whole lattices: a lattice held as two halves opens a
// cluster pair (one half at the start of each block), one longer than one block (more
// than NT threads) opens a pair as a ring across both blocks; the others fill the
// pairs' spare threads first, then blocks of NT threads.
inline void pack_rings(std::vector<Piece>& pieces, int NT, Bins* blocks, Bins* pairs) {
  blocks->cap = NT;
  pairs->cap = 2 * NT;
  pairs->pair = true;
  for (size_t i = 0; i + 1 < pieces.size(); ++i) {
    if (pieces[i].halo == 0) continue;
    pieces[i].t0 = 0;
    pieces[i + 1].t0 = NT;
    pairs->add({(int)i, (int)i + 1}, pieces[i].nthr, NT + pieces[i + 1].nthr);
    ++i;
  }
  for (int i : by_threads_desc(pieces)) {
    if (pieces[i].halo > 0) continue;
    if (pieces[i].nthr > NT) {
      pieces[i].t0 = 0;
      pairs->add({i}, NT, pieces[i].nthr);
    } else if (!pairs->first_fit(pieces, i) && !blocks->first_fit(pieces, i)) {
      blocks->open(pieces, i);
    }
  }
  pairs->key.resize(pairs->used.size());
  for (size_t b = 0; b < pairs->used.size(); ++b) pairs->key[b] = pairs->used0[b] + pairs->used[b] - NT;
}

// One queue for every whole lattice: the single-block bundles go two to a cluster
// pair (the second one's pieces shifted by NT threads, so no piece spans the block
// edge and its blocks never wait on each other), queued after the pair bundles whose
// piece spans the edge; within each kind, largest first.
// (Groups appended here take no further pieces.)
inline void merge_blocks_into_pairs(std::vector<Piece>& pieces, int NT, const Bins& blocks, Bins* pairs) {
  pairs->cap = 2 * NT;
  for (size_t b = 0; b < pairs->key.size(); ++b) pairs->key[b] += 4 * NT;
  const std::vector<int> order = stable_desc(blocks.used);
  for (size_t q = 0; q < order.size(); q += 2) {
    const size_t a = (size_t)order[q];
    const size_t g = pairs->new_group(blocks.used[a], q + 1 < order.size() ? NT + blocks.used[(size_t)order[q + 1]]
                                                                           : blocks.used[a]);
    for (int i = blocks.head[a]; i >= 0; i = blocks.nxt[(size_t)i]) pairs->link(g, i);
    if (q + 1 < order.size()) {
      const size_t c = (size_t)order[q + 1];
      for (int i = blocks.head[c]; i >= 0; i = blocks.nxt[(size_t)i]) {
        pieces[(size_t)i].t0 += NT;
        pairs->link(g, i);
      }
    }
    pairs->key.push_back(blocks.used[a]);  // the fuller of the two blocks
  }
}

inline void pack_blocks(std::vector<Piece>& pieces, int NT, Bins* blocks) {
  blocks->cap = NT;
  for (int i : by_threads_desc(pieces))
    if (!blocks->first_fit(pieces, i)) blocks->open(pieces, i);
}

}  // namespace plan
}  // namespace lbks
