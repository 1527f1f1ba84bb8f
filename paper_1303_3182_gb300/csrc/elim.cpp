// Elimination lists of tiled QR (Section 3.2).  Host code, integer-exact.
//
// Every generator returns the list in canonical order: by panel column, then by the
// time step / tree level inside the column, then by row.  Rows are 0-based.
#include <algorithm>
#include <map>
#include <set>
#include <tuple>

#include "tqr_internal.h"

namespace tqr {
namespace {

int trailing_zeros(int d) {
  int n = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++n;
  }
  return n;
}

// FlatTree / Sameh-Kuck (Section 3.2.1): the diagonal row zeroes its column top-down.
void flat(int p, int q, std::vector<Elim> &out) {
  for (int k = 0; k < std::min(p, q); ++k)
    for (int i = k + 1; i < p; ++i) out.push_back({k, i, k});
}

// PlasmaTree(bs) (Section 3.2.4): flat inside domains of bs rows counted from the
// diagonal, then a binary merge of the domain heads (head d at level v2(d) by head
// d - 2^v2(d)).  bs = 1 is BinaryTree, bs >= p is FlatTree.
void plasma(int p, int q, int bs, std::vector<Elim> &out) {
  for (int k = 0; k < std::min(p, q); ++k) {
    std::vector<int> heads;
    for (int h = k; h < p; h += bs) heads.push_back(h);
    for (int h : heads)
      for (int i = h + 1; i < std::min(h + bs, p); ++i) out.push_back({k, i, h});
    std::vector<std::tuple<int, int, int, int>> merge;  // level, d, row, pivot
    for (int d = 1; d < static_cast<int>(heads.size()); ++d) {
      const int l = trailing_zeros(d);
      merge.emplace_back(l, d, heads[d], heads[d - (1 << l)]);
    }
    std::sort(merge.begin(), merge.end());
    for (auto &m : merge) out.push_back({k, std::get<2>(m), std::get<3>(m)});
  }
}

// Fibonacci scheme of order 1 (Modi-Clarke; Section 3.2.1).  In column 1 (thesis
// numbering) row r >= 2 is zeroed at step x - y + 1 with x minimal s.t. x(x+1)/2 >= p-1
// and y minimal s.t. r <= y(y+1)/2 + 1; column k is column 1 moved down k-1 rows and
// 2(k-1) steps later; a run of z rows zeroed at one step uses the z rows above it.
void fibonacci(int p, int q, std::vector<Elim> &out) {
  int x = 0;
  while (x * (x + 1) / 2 < p - 1) ++x;
  auto step1 = [&](int r) {
    int y = 0;
    while (r > y * (y + 1) / 2 + 1) ++y;
    return x - y + 1;
  };
  for (int k = 0; k < std::min(p, q); ++k) {
    std::map<int, std::vector<int>> runs;  // step -> rows
    for (int i = k + 1; i < p; ++i) runs[step1(i - k + 1) + 2 * k].push_back(i);
    for (auto &kv : runs) {
      const int z = static_cast<int>(kv.second.size());
      for (int i : kv.second) out.push_back({k, i, i - z});
    }
  }
}

// Greedy (Section 3.2.1 / Algorithm "tiled-greedy"): at each coarse step, in every
// column, the live rows (not yet zeroed here, zeroed in the previous column at an
// earlier step) lose their bottom half to the rows right above.
void greedy(int p, int q, std::vector<Elim> &out) {
  const int kmax = std::min(p, q);
  std::vector<std::vector<int>> zstep(kmax, std::vector<int>(p, 0));  // 0 = not zeroed
  std::vector<std::vector<std::tuple<int, int, int>>> cols(kmax);      // step, row, piv
  int64_t remaining = 0;
  for (int k = 0; k < kmax; ++k) remaining += p - 1 - k;
  for (int s = 1; remaining > 0; ++s) {
    for (int k = 0; k < kmax; ++k) {
      std::vector<int> live;
      for (int i = k; i < p; ++i) {
        if (zstep[k][i]) continue;
        if (k > 0 && !(zstep[k - 1][i] && zstep[k - 1][i] <= s - 1)) continue;
        live.push_back(i);
      }
      const int n = static_cast<int>(live.size()), h = n / 2;
      for (int j = 0; j < h; ++j) {
        const int i = live[n - h + j], piv = live[n - 2 * h + j];
        cols[k].emplace_back(s, i, piv);
        zstep[k][i] = s;
        --remaining;
      }
    }
  }
  for (int k = 0; k < kmax; ++k) {
    std::sort(cols[k].begin(), cols[k].end());
    for (auto &e : cols[k]) out.push_back({k, std::get<1>(e), std::get<2>(e)});
  }
}

// ASAP on one column (Section 3.2.2, Definition "optiter" with weight 2): at every
// event time the rows that are triangularized, not zeroed and not busy are ready; with
// n >= 2 of them, the bottom 2*floor(n/2) are paired, the lower half zeroed by the upper
// half in order; a pivot is busy for one TTQRT (2 units).
std::vector<Elim> asap_column(int p, int k, const std::vector<int64_t> &ready) {
  const int nrow = p - k;
  std::vector<char> zeroed(nrow, 0);
  std::vector<int64_t> busy(nrow, 0);
  std::set<int64_t> events(ready.begin(), ready.end());
  std::vector<Elim> out;
  int nzero = 0;
  while (nzero < nrow - 1 && !events.empty()) {
    const int64_t t = *events.begin();
    events.erase(events.begin());
    std::vector<int> avail;
    for (int r = 0; r < nrow; ++r)
      if (!zeroed[r] && ready[r] <= t && busy[r] <= t) avail.push_back(r);
    const int n = static_cast<int>(avail.size());
    if (n < 2) continue;
    const int s = n / 2;
    std::vector<std::pair<int, int>> started;  // row, pivot
    for (int j = 0; j < s; ++j) {
      const int piv = avail[n - 2 * s + j], row = avail[n - s + j];
      started.emplace_back(row, piv);
      zeroed[row] = 1;
      busy[piv] = t + kWTtqrt;
      ++nzero;
    }
    std::sort(started.begin(), started.end());
    for (auto &e : started) out.push_back({k, k + e.first, k + e.second});
    events.insert(t + kWTtqrt);
  }
  return out;
}

// GrASAP(n_asap) (Definition "grasap"): Greedy on the first q - n_asap columns and
// ASAP, driven by the simulated finish times of GEQRT, on the rest.  GrASAP = GrASAP(1);
// ASAP = GrASAP(q); when p <= q the last column zeroes nothing and Greedy is used.
void grasap(int p, int q, int n_asap, std::vector<Elim> &out) {
  const int kmax = std::min(p, q);
  std::vector<Elim> gl;
  greedy(p, q, gl);
  int first_asap = (p > q) ? q - n_asap : kmax;
  if (n_asap >= q) first_asap = 0;
  std::vector<std::vector<Elim>> by_col(kmax);
  for (const Elim &e : gl) by_col[e.k].push_back(e);
  GraphBuilder b(p * q * kRegionsPerTile);
  for (int k = 0; k < kmax; ++k) {
    std::vector<int> gid = add_panel_tasks(b, p, q, k);
    std::vector<Elim> col;
    if (k < first_asap) {
      col = by_col[k];
    } else {
      std::vector<int64_t> ready(gid.size());
      for (size_t r = 0; r < gid.size(); ++r) ready[r] = b.finish[gid[r]];
      col = asap_column(p, k, ready);
    }
    add_elim_tasks(b, q, k, col);
    out.insert(out.end(), col.begin(), col.end());
  }
}

}  // namespace

bool elimination_list(int p, int q, int tree, int bs, std::vector<Elim> &out) {
  out.clear();
  switch (tree) {
    case 0: flat(p, q, out); return true;
    case 1: plasma(p, q, bs, out); return true;
    case 2: plasma(p, q, 1, out); return true;
    case 3: fibonacci(p, q, out); return true;
    case 4: greedy(p, q, out); return true;
    case 5: grasap(p, q, 1, out); return true;
    case 6: grasap(p, q, q, out); return true;
    default: return false;
  }
}

}  // namespace tqr
