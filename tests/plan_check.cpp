// Host check of the resident kernel's planning (paper_1711_03540_gb300/csrc/lbks_plan.h),
// built and run by tests/test_plan_host.py.  Reads one case per line on stdin:
//     C S NT cl kx kseg merge N_0 N_1 ... N_{n-1}
// (c_max, sites per thread, threads per block, blocks per work group of whole
// lattices, steps between halo exchanges of halves (0: none), steps per segment launch,
// 1 to put single-block bundles two to a pair) and prints one line per case:
//     OK rings=<pieces> halves=<lattices> spans=<rings across a pair> segs=<pieces> blocks=<groups>
//        pairs=<groups> segblocks=<groups> ring_threads=<threads> seg_threads=<threads>
// or FAIL <reason>.  The line "PLAIN <SMs> <reservoir 0|1> <c_max> N_0 ... N_{n-1}" checks
// the plain family's tiles (every site, ghosts of reservoir lattices included, in
// exactly one tile of its run; lengths within the chosen tile size; the size the
// largest of 256, 128, 64, 32 giving two tiles per SM, else 32) and prints
//     OK tile=<sites> tiles=<count>
// The line "FIRSTFIT <trials> <seed>" compares the groups' first
// fit with a linear scan of the groups on random pieces; "ORDER <trials> <seed>" the
// counting sort that orders pieces and bundles with a stable sort.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <iostream>
#include <random>
#include <sstream>
#include <string>
#include <vector>

#include "lbks_plan.h"

using lbks::Piece;
using namespace lbks::plan;

namespace {

std::string fail_;

bool check(bool ok, const std::string& why) {
  if (!ok && fail_.empty()) fail_ = why;
  return ok;
}

// Each piece: V threads hold S or S-1 sites, V (S - 1) < n <= V S.
void check_piece_shape(const Piece& p, int S) {
  const int64_t V = p.nthr;
  check(V >= 1 && p.n > V * (S - 1) && p.n <= V * S, "piece does not split into runs of S and S-1 sites");
  check(p.st_lo >= 0 && p.st_lo < p.st_hi && p.st_hi <= p.n, "stored range outside the piece");
}

// Every site of every run is stored by exactly one piece.
void check_coverage(const std::vector<int64_t>& Ns, const std::vector<Piece>& all) {
  std::vector<std::vector<int>> hits(Ns.size());
  for (size_t r = 0; r < Ns.size(); ++r) hits[r].assign((size_t)Ns[r], 0);
  for (const Piece& p : all) {
    if (!check(p.run >= 0 && p.run < (int)Ns.size(), "piece of an unknown run")) return;
    const int64_t N = Ns[p.run];
    for (int li = p.st_lo; li < p.st_hi; ++li) ++hits[p.run][(size_t)((p.x0 + li) % N)];
  }
  for (size_t r = 0; r < Ns.size(); ++r)
    for (int64_t x = 0; x < Ns[r]; ++x)
      if (hits[r][(size_t)x] != 1) {
        check(false, "run " + std::to_string(r) + " site " + std::to_string(x) + " stored " +
                         std::to_string(hits[r][(size_t)x]) + " times");
        return;
      }
}

// Groups: thread ranges of their pieces inside the group and disjoint; in pair groups a
// piece lies in one block unless it is the one ring across both (t0 = 0, more than NT
// threads); halves sit at thread 0 of block 0 and block 1.
void check_groups(const Bins& g, const std::vector<Piece>& pieces, int NT, bool pair, std::vector<int>* seen) {
  for (size_t b = 0; b < g.groups(); ++b) {
    std::vector<char> used((size_t)(pair ? 2 * NT : NT), 0);
    int spans = 0, halves = 0;
    for (int i : g.members(b)) {
      const Piece& p = pieces[(size_t)i];
      ++(*seen)[(size_t)i];
      const int lo = p.t0, hi = p.t0 + p.nthr;
      if (!check(lo >= 0 && hi <= (pair ? 2 * NT : NT), "piece outside its group")) return;
      if (pair && lo < NT && hi > NT) {
        ++spans;
        check(lo == 0 && p.halo == 0, "a piece other than a whole ring spans the block edge");
      }
      if (p.halo > 0) {
        ++halves;
        check(lo == 0 || lo == NT, "a half does not start at thread 0 of its block");
      }
      for (int t = lo; t < hi; ++t) {
        if (!check(!used[(size_t)t], "two pieces share a thread")) return;
        used[(size_t)t] = 1;
      }
    }
    check(spans <= 1, "more than one piece spans the block edge");
    check(halves == 0 || (halves == 2 && spans == 0), "halves not in pairs, or beside a spanning ring");
  }
}

}  // namespace

namespace {

std::string run_case(int C, int S, int NT, int cl, int kx, int kseg, int merge, const std::vector<int64_t>& Ns) {
  fail_.clear();
  std::vector<Piece> rings, segs;
  if (!plan_pieces(Ns, C, S, NT, cl * NT, kseg, kx, &rings, &segs)) return "FAIL plan_pieces: a run cannot be held";
  for (const Piece& p : rings) check_piece_shape(p, S);
  for (const Piece& p : segs) check_piece_shape(p, S);
  // halos: halves refreshed every kx steps need c_max kx sites each side; segments run
  // kseg steps per launch and need c_max kseg
  for (const Piece& p : rings)
    if (p.halo > 0)
      check(kx > 0 && p.halo == C * kx && p.st_lo == p.halo && p.n - p.st_hi >= p.halo, "half with a short halo");
  for (const Piece& p : segs)
    check(p.st_lo == C * kseg && p.n - p.st_hi >= C * kseg && p.halo == 0, "segment with a short halo");
  std::vector<Piece> all = rings;
  all.insert(all.end(), segs.begin(), segs.end());
  check_coverage(Ns, all);

  Bins blocks, pairs, segbins;
  pack_rings(rings, NT, &blocks, &pairs);
  if (cl == 1) check((pairs.groups() == 0), "pair groups with one-block work groups");
  const size_t nsingle = blocks.groups(), npair = pairs.groups();
  const bool merged = merge && npair && nsingle;
  if (merged) {
    merge_blocks_into_pairs(rings, NT, blocks, &pairs);
    blocks = Bins{};
  }
  pack_blocks(segs, NT, &segbins);
  std::vector<int> seen_r(rings.size(), 0), seen_s(segs.size(), 0);
  check_groups(blocks, rings, NT, false, &seen_r);
  check_groups(pairs, rings, NT, true, &seen_r);
  check_groups(segbins, segs, NT, false, &seen_s);
  for (int v : seen_r) check(v == 1, "a ring or half is not in exactly one group");
  for (int v : seen_s) check(v == 1, "a segment is not in exactly one group");
  // bundles as uploaded: pieces of each group contiguous, groups largest first
  std::vector<Piece> ordered;
  std::vector<int2> bundles;
  pairs.emit(rings, &ordered, &bundles);
  size_t total = 0;
  for (const int2& b : bundles) total += (size_t)b.y;
  check(total == ordered.size(), "bundles do not cover the ordered pieces");
  if (merged) check(pairs.groups() == npair + (nsingle + 1) / 2, "single-block groups not two to a pair");
  if (!fail_.empty()) return "FAIL " + fail_;
  int halves = 0, spans = 0;
  int64_t ring_threads = 0, seg_threads = 0;
  for (const Piece& p : rings) {
    halves += p.halo > 0 ? 1 : 0;
    spans += p.nthr > NT ? 1 : 0;
    ring_threads += p.nthr;
  }
  for (const Piece& p : segs) seg_threads += p.nthr;
  std::ostringstream o;
  o << "OK rings=" << rings.size() << " halves=" << halves / 2 << " spans=" << spans << " segs=" << segs.size()
    << " blocks=" << blocks.groups() << " pairs=" << pairs.groups() << " segblocks=" << segbins.groups()
    << " ring_threads=" << ring_threads << " seg_threads=" << seg_threads;
  return o.str();
}

// The former linear first fit, the reference for the segment-tree search.
struct LinearFit {
  int cap = 0;
  bool pair = false;
  std::vector<int> used, used0;
  int fit(int need) {
    for (size_t b = 0; b < used.size(); ++b) {
      if (pair && used0[b] + need <= cap / 2) { used0[b] += need; return (int)b; }
      if (used[b] + need <= cap) { used[b] += need; return (int)b; }
    }
    return -1;
  }
};

std::string first_fit_trials(int trials, unsigned seed) {
  std::mt19937 rng(seed);
  for (int trial = 0; trial < trials; ++trial) {
    const int NT = 32 * (2 + (int)(rng() % 15));
    const bool pair = trial % 2;
    Bins B;
    B.cap = pair ? 2 * NT : NT;
    B.pair = pair;
    LinearFit L;
    L.cap = B.cap;
    L.pair = pair;
    const int n = 1 + (int)(rng() % 3000);
    std::vector<Piece> pieces((size_t)n);
    for (int i = 0; i < n; ++i) {
      pieces[(size_t)i] = Piece{};
      pieces[(size_t)i].nthr = 1 + (int)(rng() % (unsigned)NT);
      if (pair && rng() % 5 == 0) {  // a group opened by a half pair or a spanning ring
        const int u0 = (int)(rng() % (unsigned)(NT + 1)), u = NT + (int)(rng() % (unsigned)(NT + 1));
        B.add({}, u0, u);
        L.used.push_back(u);
        L.used0.push_back(u0);
      }
      const size_t before = B.used.size();
      const bool fb = B.first_fit(pieces, i);
      const int fl = L.fit(pieces[(size_t)i].nthr);
      if (fb != (fl >= 0)) return "FAIL first fit: tree and scan disagree on whether a piece fits";
      if (fb && (B.used != L.used || (pair && B.used0 != L.used0)))
        return "FAIL first fit: tree and scan chose different groups";
      if (!fb) {
        if (pair) {
          B.add({i}, pieces[(size_t)i].nthr, NT);
          L.used.push_back(NT);
          L.used0.push_back(pieces[(size_t)i].nthr);
        } else {
          B.open(pieces, i);
          L.used.push_back(pieces[(size_t)i].nthr);
        }
      }
      (void)before;
    }
  }
  return "OK first fit identical to the scan in " + std::to_string(trials) + " trials";
}

// stable_desc (counting) against std::stable_sort on random keys with many ties.
std::string order_trials(int trials, unsigned seed) {
  std::mt19937 rng(seed);
  for (int t = 0; t < trials; ++t) {
    const int n = (int)(rng() % 3000), kmax = 1 + (int)(rng() % 1200);
    std::vector<int> k(n);
    for (int& v : k) v = (int)(rng() % (unsigned)kmax);
    std::vector<int> ref(n);
    for (int i = 0; i < n; ++i) ref[i] = i;
    std::stable_sort(ref.begin(), ref.end(), [&](int a, int b) { return k[a] > k[b]; });
    if (stable_desc(k) != ref) return "FAIL stable_desc differs from a stable sort";
  }
  return "OK";
}

}  // namespace

// The plain family's tiles for one set of runs.
std::string plain_case(int sms, bool reservoir, int C, const std::vector<int64_t>& Ns) {
  fail_.clear();
  int tile = 0;
  const std::vector<lbks::Tile> pt = plain_tiles(Ns, reservoir, C, sms, &tile);
  check(tile == 32 || tile == 64 || tile == 128 || tile == 256, "tile size not a power of two in [32, 256]");
  auto count = [&](int t) {
    int64_t n = 0;
    for (int64_t N : Ns) n += (N + (reservoir ? 2 * C : 0) + t - 1) / t;
    return n;
  };
  check(tile == 32 || count(tile) >= 2 * (int64_t)sms, "fewer than two tiles per SM above the smallest size");
  check(tile == 256 || count(2 * tile) < 2 * (int64_t)sms, "a larger tile would still give two tiles per SM");
  std::vector<std::vector<int>> hits(Ns.size());
  for (size_t r = 0; r < Ns.size(); ++r) hits[r].assign((size_t)(Ns[r] + (reservoir ? 2 * C : 0)), 0);
  const int64_t g0 = reservoir ? -C : 0;
  for (const lbks::Tile& t : pt) {
    if (!check(t.run >= 0 && t.run < (int)Ns.size(), "tile of an unknown run")) break;
    check(t.len >= 1 && t.len <= tile, "tile length outside [1, tile size]");
    for (int k = 0; k < t.len; ++k) {
      const int64_t x = (int64_t)t.x0 + k - g0;
      if (!check(x >= 0 && x < (int64_t)hits[t.run].size(), "tile outside its run")) break;
      ++hits[t.run][(size_t)x];
    }
  }
  for (size_t r = 0; r < Ns.size() && fail_.empty(); ++r)
    for (int h : hits[r])
      if (!check(h == 1, "run " + std::to_string(r) + ": a site in " + std::to_string(h) + " tiles")) break;
  if (!fail_.empty()) return "FAIL " + fail_;
  return "OK tile=" + std::to_string(tile) + " tiles=" + std::to_string(pt.size());
}

int main() {
  std::string line;
  while (std::getline(std::cin, line)) {
    if (line.empty()) continue;
    std::istringstream in(line);
    std::string head;
    in >> head;
    if (head == "FIRSTFIT") {
      int trials = 0;
      unsigned seed = 0;
      in >> trials >> seed;
      std::cout << first_fit_trials(trials, seed) << "\n";
      continue;
    }
    if (head == "PLAIN") {
      int sms = 0, res = 0, C = 0;
      in >> sms >> res >> C;
      std::vector<int64_t> Ns;
      int64_t v;
      while (in >> v) Ns.push_back(v);
      std::cout << plain_case(sms, res != 0, C, Ns) << "\n";
      continue;
    }
    if (head == "ORDER") {
      int trials = 0;
      unsigned seed = 0;
      in >> trials >> seed;
      std::cout << order_trials(trials, seed) << "\n";
      continue;
    }
    const int C = std::atoi(head.c_str());
    int S = 0, NT = 0, cl = 0, kx = 0, kseg = 0, merge = 0;
    in >> S >> NT >> cl >> kx >> kseg >> merge;
    std::vector<int64_t> Ns;
    int64_t v;
    while (in >> v) Ns.push_back(v);
    std::cout << run_case(C, S, NT, cl, kx, kseg, merge, Ns) << "\n";
  }
  return 0;
}
