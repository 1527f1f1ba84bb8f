// Tile task graph of the TT tiled QR (Section 3.1.1, Algorithm "elimTR"; dependencies
// Eq. ttdeps and ttdeps2) and its executor order.
//
// The graph is the sequential column-by-column program - for every panel k: GEQRT(i,k)
// and UNMQR(i,k,j) for all rows i >= k, then TTQRT(i,piv,k) and TTMQR(i,piv,k,j) for
// each elimination of column k in list order - with a dependency wherever two kernels
// touch the same tile region and one of them writes it.  Splitting each panel tile into
// its strictly-lower part (GEQRT reflectors, read by UNMQR) and its upper part (R and
// later the TTQRT reflectors) lets UNMQR overlap TTQRT as Section 3.1.1 states.
#include <algorithm>
#include <functional>
#include <map>
#include <numeric>
#include <queue>

#include "tqr_internal.h"

namespace tqr {

GraphBuilder::GraphBuilder(int nregions)
    : last_writer(nregions, -1), readers(nregions) {}

int GraphBuilder::add(const Task &t, int w, const int *reads, int nr, const int *writes,
                      int nw) {
  const int id = static_cast<int>(tasks.size());
  std::vector<int32_t> pr;
  for (int a = 0; a < nr; ++a) {
    const int r = reads[a];
    if (last_writer[r] >= 0) pr.push_back(last_writer[r]);
  }
  for (int a = 0; a < nw; ++a) {
    const int r = writes[a];
    if (last_writer[r] >= 0) pr.push_back(last_writer[r]);
    for (int32_t x : readers[r]) pr.push_back(x);
  }
  std::sort(pr.begin(), pr.end());
  pr.erase(std::unique(pr.begin(), pr.end()), pr.end());
  int64_t start = 0;
  for (int32_t x : pr) start = std::max(start, finish[x]);
  for (int a = 0; a < nr; ++a) readers[reads[a]].push_back(id);
  for (int a = 0; a < nw; ++a) {
    last_writer[writes[a]] = id;
    readers[writes[a]].clear();
  }
  tasks.push_back(t);
  weight.push_back(w);
  finish.push_back(start + w);
  preds.push_back(std::move(pr));
  return id;
}

namespace {
// Region id lists of the task kinds: the whole upper part of a tile is its row blocks.
struct Regions {
  int r[16];
  int n = 0;
  void add(int x) { r[n++] = x; }
  void L(int q, int i, int j) { add(region_L(q, i, j)); }
  void U(int q, int i, int j) {
    for (int bb = 0; bb < kPanelSplits; ++bb) add(region_Ub(q, i, j, bb));
  }
  void tile(int q, int i, int j) {
    L(q, i, j);
    U(q, i, j);
  }
  void cps(int q, int i, int j) {
    for (int c = 0; c < kColParts; ++c) add(region_cp(q, i, j, c));
  }
};
}  // namespace

std::vector<int> add_panel_tasks(GraphBuilder &b, int p, int q, int k, const char *square, bool prep,
                                 int colparts) {
  std::vector<int> geqrt_ids;
  for (int i = k; i < p; ++i) {
    if (square && square[i]) {
      geqrt_ids.push_back(-1);
      continue;
    }
    Regions w;
    w.tile(q, i, k);
    if (colparts > 1) w.cps(q, i, k);
    geqrt_ids.push_back(b.add(Task{kGeqrt, i, -1, (int16_t)k, -1}, kWGeqrt, nullptr, 0, w.r, w.n));
    if (prep) {
      const int rd[1] = {region_L(q, i, k)};
      const int wr[1] = {region_ops(q, i, k, 0)};
      b.add(Task{kPrepG, i, -1, (int16_t)k, -1}, 0, rd, 1, wr, 1);
    }
    for (int j = k + 1; j < q; ++j) {
      const int rd[2] = {region_L(q, i, k), region_ops(q, i, k, 0)};
      if (colparts > 1) {
        for (int c = 0; c < colparts; ++c) {
          const int wr[1] = {region_cp(q, i, j, c)};
          b.add(Task{kUnmqr, i, -1, (int16_t)k, (int16_t)(j | (c << kColShift))}, kWUnmqr, rd, 1, wr, 1);
        }
        continue;
      }
      Regions wj;
      wj.tile(q, i, j);
      b.add(Task{kUnmqr, i, -1, (int16_t)k, (int16_t)j}, kWUnmqr, rd, prep ? 2 : 1, wj.r, wj.n);
    }
  }
  return geqrt_ids;
}

void add_elim_tasks(GraphBuilder &b, int q, int k, const std::vector<Elim> &col, const char *square, bool prep,
                    bool split, int colparts) {
  for (const Elim &e : col) {
    const bool ts = square && square[e.i];
    if (split) {
      // block bb writes row block bb of the pivot's R and the zeroed tile (its later
      // columns): blocks of one elimination run in order, and block bb of the next
      // elimination on the same pivot waits only for block bb of this one
      for (int bb = 0; bb < kPanelSplits; ++bb) {
        Regions w;
        w.add(region_Ub(q, e.piv, k, bb));
        if (ts)
          w.tile(q, e.i, k);
        else
          w.U(q, e.i, k);
        b.add(Task{ts ? kTsqrtS : kTtqrtS, e.i, e.piv, (int16_t)k, (int16_t)bb}, ts ? 2 : 1, nullptr, 0, w.r, w.n);
      }
    } else {
      // TSQRT overwrites the whole square tile (i,k) with its reflectors; TTQRT its upper part
      Regions w;
      w.U(q, e.piv, k);
      if (ts)
        w.tile(q, e.i, k);
      else
        w.U(q, e.i, k);
      if (colparts > 1) {
        w.cps(q, e.piv, k);
        w.cps(q, e.i, k);
      }
      b.add(Task{ts ? kTsqrt : kTtqrt, e.i, e.piv, (int16_t)k, -1}, ts ? kWTsqrt : kWTtqrt, nullptr, 0, w.r, w.n);
    }
    if (prep) {
      Regions rd;
      if (ts)
        rd.tile(q, e.i, k);
      else
        rd.U(q, e.i, k);
      const int wr[1] = {region_ops(q, e.i, k, 1)};
      // j carries the kernel: 1 = TSQRT (dense reflector tile), 0 = TTQRT
      b.add(Task{kPrepT, e.i, e.piv, (int16_t)k, (int16_t)(ts ? 1 : 0)}, 0, rd.r, rd.n, wr, 1);
    }
    for (int j = k + 1; j < q; ++j) {
      Regions rd;
      if (ts)
        rd.tile(q, e.i, k);
      else
        rd.U(q, e.i, k);
      if (prep) rd.add(region_ops(q, e.i, k, 1));
      if (colparts > 1) {
        for (int c = 0; c < colparts; ++c) {
          const int wr[2] = {region_cp(q, e.piv, j, c), region_cp(q, e.i, j, c)};
          b.add(Task{ts ? kTsmqr : kTtmqr, e.i, e.piv, (int16_t)k, (int16_t)(j | (c << kColShift))},
                ts ? kWTsmqr : kWTtmqr, rd.r, rd.n, wr, 2);
        }
        continue;
      }
      Regions w4;
      w4.tile(q, e.piv, j);
      w4.tile(q, e.i, j);
      b.add(Task{ts ? kTsmqr : kTtmqr, e.i, e.piv, (int16_t)k, (int16_t)j}, ts ? kWTsmqr : kWTtmqr, rd.r, rd.n, w4.r,
            w4.n);
    }
  }
}

std::vector<int64_t> backflow_priorities(const std::vector<std::vector<int32_t>> &succ,
                                         const std::vector<int64_t> &w) {
  const int n = static_cast<int>(w.size());
  std::vector<int64_t> cp(n, 0);
  for (int t = n - 1; t >= 0; --t) {  // program order is topological
    int64_t best = 0;
    for (int32_t s : succ[t]) best = std::max(best, cp[s]);
    cp[t] = best + w[t];
  }
  return cp;
}

int64_t cp_list_schedule(const std::vector<std::vector<int32_t>> &succ, const std::vector<int32_t> &npred,
                         const std::vector<int64_t> &w, const std::vector<int64_t> &prio, int nproc,
                         std::vector<int64_t> *start) {
  const int n = static_cast<int>(w.size());
  using Item = std::pair<int64_t, int32_t>;
  // ready tasks: largest priority first, then the earlier task of the program
  auto later = [](const Item &a, const Item &c) { return a.first != c.first ? a.first < c.first : a.second > c.second; };
  std::priority_queue<Item, std::vector<Item>, decltype(later)> ready(later);
  std::priority_queue<Item, std::vector<Item>, std::greater<Item>> running;  // (finish, task)
  std::vector<int32_t> missing(npred);
  for (int t = 0; t < n; ++t)
    if (missing[t] == 0) ready.push({prio[t], t});
  if (start) start->assign(n, 0);
  int free = nproc, done = 0;
  int64_t now = 0, makespan = 0;
  while (done < n) {
    while (free > 0 && !ready.empty()) {
      const int32_t t = ready.top().second;
      ready.pop();
      if (start) (*start)[t] = now;
      running.push({now + w[t], t});
      makespan = std::max(makespan, now + w[t]);
      --free;
    }
    now = running.top().first;
    while (!running.empty() && running.top().first == now) {
      const int32_t t = running.top().second;
      running.pop();
      ++free;
      ++done;
      for (int32_t s : succ[t])
        if (--missing[s] == 0) ready.push({prio[s], s});
    }
  }
  return makespan;
}

int64_t alap_derived_bound(const std::vector<int64_t> &w, const std::vector<int64_t> &prio, int nproc,
                           int64_t *lost) {
  // every task as late as possible on unbounded processors: t runs over
  // [crit - prio[t], crit - prio[t] + w[t])
  int64_t crit = 0, tseq = 0;
  for (size_t t = 0; t < w.size(); ++t) {
    crit = std::max(crit, prio[t]);
    tseq += w[t];
  }
  std::map<int64_t, int64_t> delta;
  for (size_t t = 0; t < w.size(); ++t) {
    delta[crit - prio[t]] += 1;
    delta[crit - prio[t] + w[t]] -= 1;
  }
  // active count per segment, then the idle area of nproc processors walking back from
  // the end until more than nproc tasks are active
  std::vector<std::pair<int64_t, int64_t>> seg;  // (length, active)
  int64_t active = 0;
  for (auto it = delta.begin(); it != delta.end(); ++it) {
    active += it->second;
    auto nx = std::next(it);
    if (nx != delta.end()) seg.push_back({nx->first - it->first, active});
  }
  int64_t la = 0;
  for (auto it = seg.rbegin(); it != seg.rend(); ++it) {
    if (it->second > nproc) break;
    la += (nproc - it->second) * it->first;
  }
  if (lost) *lost = la;
  const int64_t tp = (tseq + la + nproc - 1) / nproc;
  return std::max(crit, tp);
}

void finalize_graph(GraphBuilder &b, Graph &g, int64_t drop_edge, const OrderSpec *spec) {
  const int n = static_cast<int>(b.tasks.size());
  // successors in program order
  std::vector<std::vector<int32_t>> succ(n);
  for (int t = 0; t < n; ++t)
    for (int32_t x : b.preds[t]) succ[x].push_back(t);
  // longest path to a sink, including the task itself (thesis weights)
  const std::vector<int64_t> wt(b.weight.begin(), b.weight.end());
  const std::vector<int64_t> bottom = backflow_priorities(succ, wt);
  std::vector<int32_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  if (spec && spec->mode == 1) {
    // start times of the bounded-processor CP-method schedule with the given kind
    // weights (all positive): a task starts after its predecessors finished, so this
    // order is topological
    std::vector<int64_t> w(n);
    std::vector<int32_t> npred(n);
    for (int t = 0; t < n; ++t) {
      w[t] = spec->w[b.tasks[t].kind];
      npred[t] = static_cast<int32_t>(b.preds[t].size());
    }
    const std::vector<int64_t> prio = backflow_priorities(succ, w);
    std::vector<int64_t> st;
    cp_list_schedule(succ, npred, w, prio, std::max(1, spec->nproc), &st);
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t c) {
      if (st[a] != st[c]) return st[a] < st[c];
      if (prio[a] != prio[c]) return prio[a] > prio[c];
      return a < c;
    });
  } else {
    // earliest start with unbounded processors, then the longer remaining path first,
    // then program order.  Earliest start strictly increases along every edge, so this
    // order is topological.
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t c) {
      const int64_t sa = b.finish[a] - b.weight[a], sc = b.finish[c] - b.weight[c];
      if (sa != sc) return sa < sc;
      if (bottom[a] != bottom[c]) return bottom[a] > bottom[c];
      return a < c;
    });
  }
  std::vector<int32_t> pos(n);
  for (int r = 0; r < n; ++r) pos[order[r]] = r;

  g.tasks.resize(n);
  g.weight.resize(n);
  g.start.resize(n);
  g.bottom.resize(n);
  g.indeg.assign(n, 0);
  g.succ_ptr.assign(n + 1, 0);
  g.succ_idx.clear();
  g.critical_path = 0;
  for (int c = 0; c < 4; ++c) g.counts[c] = 0;
  for (int r = 0; r < n; ++r) {
    const int t = order[r];
    g.tasks[r] = b.tasks[t];
    g.weight[r] = b.weight[t];
    g.start[r] = b.finish[t] - b.weight[t];
    g.bottom[r] = bottom[t];
    g.indeg[r] = static_cast<int32_t>(b.preds[t].size());
    g.critical_path = std::max<int64_t>(g.critical_path, b.finish[t]);
    const int kind = b.tasks[t].kind;
    if (kind >= 0 && kind < kNumKinds) g.counts[kind]++;
  }
  int64_t edge = 0;
  for (int r = 0; r < n; ++r) {
    const int t = order[r];
    std::vector<int32_t> s;
    for (int32_t x : succ[t]) s.push_back(pos[x]);
    std::sort(s.begin(), s.end());
    for (int32_t x : s) {
      // test hook: leave out one release so that its successor can never start
      if (edge++ == drop_edge) continue;
      g.succ_idx.push_back(x);
    }
    g.succ_ptr[r + 1] = static_cast<int32_t>(g.succ_idx.size());
  }
}

std::vector<std::vector<char>> ts_square_rows(int p, int q, const std::vector<Elim> &elims) {
  const int kmax = std::min(p, q);
  std::vector<std::vector<char>> pivot(kmax, std::vector<char>(p, 0)), square(kmax, std::vector<char>(p, 0));
  for (const Elim &e : elims) pivot[e.k][e.piv] = 1;
  for (const Elim &e : elims)
    if (!pivot[e.k][e.i]) square[e.k][e.i] = 1;
  return square;
}

void add_factor_program(GraphBuilder &b, int p, int q, const std::vector<Elim> &elims, bool ts, bool prep,
                        bool split, int colparts) {
  const int kmax = std::min(p, q);
  std::vector<std::vector<Elim>> by_col(kmax);
  for (const Elim &e : elims) by_col[e.k].push_back(e);
  std::vector<std::vector<char>> square;
  if (ts) square = ts_square_rows(p, q, elims);
  for (int k = 0; k < kmax; ++k) {
    const char *sq = ts ? square[k].data() : nullptr;
    add_panel_tasks(b, p, q, k, sq, prep, colparts);
    add_elim_tasks(b, q, k, by_col[k], sq, prep, split, colparts);
  }
}

void build_factor_graph(int p, int q, const std::vector<Elim> &elims, Graph &g, int64_t drop_edge,
                        const OrderSpec *order, bool ts, bool prep, bool split, int colparts) {
  GraphBuilder b(p * q * kRegionsPerTile);
  add_factor_program(b, p, q, elims, ts, prep, split, colparts);
  finalize_graph(b, g, drop_edge, order);
}

void build_applyq_graph(int p, int q, const std::vector<Elim> &elims, bool reverse, Graph &g, bool ts) {
  // Regions are the tile rows of the right-hand-side block; the factors are read-only.
  const int kmax = std::min(p, q);
  std::vector<std::vector<Elim>> by_col(kmax);
  for (const Elim &e : elims) by_col[e.k].push_back(e);
  std::vector<std::vector<char>> square;
  if (ts) square = ts_square_rows(p, q, elims);
  std::vector<Task> ops;
  for (int k = 0; k < kmax; ++k) {
    for (int i = k; i < p; ++i)
      if (!ts || !square[k][i]) ops.push_back(Task{kUnmqrB, i, -1, (int16_t)k, -1});
    for (const Elim &e : by_col[k])
      ops.push_back(Task{ts && square[k][e.i] ? kTsmqrB : kTtmqrB, e.i, e.piv, (int16_t)k, -1});
  }
  if (reverse) std::reverse(ops.begin(), ops.end());
  GraphBuilder b(p);
  for (const Task &t : ops) {
    if (t.kind == kUnmqrB) {
      const int wr[1] = {t.i};
      b.add(t, kWUnmqr, nullptr, 0, wr, 1);
    } else {
      const int wr[2] = {t.piv, t.i};
      b.add(t, t.kind == kTsmqrB ? kWTsmqr : kWTtmqr, nullptr, 0, wr, 2);
    }
  }
  finalize_graph(b, g);
}

}  // namespace tqr
