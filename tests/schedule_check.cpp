// Host check of the supernodal-solve schedules (ffa_schedule.cpp) on the factors
// of grid Laplacians: tile coverage of every block B_s, the dynamic lists
// (each node once, merged subtrees complete and children first), and the
// release protocol of the dynamic passes replayed sequentially and by racing
// threads (every task runs exactly once, after everything it depends on).
// Prints "ok" and exits 0, or prints the first violation and exits 1.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "../paper_2107_05200_gb300/csrc/ffa_factor.h"
#include "../paper_2107_05200_gb300/csrc/ffa_schedule.h"

using namespace ffa;

static int fail(const std::string& what) {
  std::printf("FAIL %s\n", what.c_str());
  return 1;
}

// 7-point (3D) or 5-point (2D) Laplacian of a grid with a positive shift, and the
// grid positions; rows in lexicographic order
static void grid_laplacian(int nx, int ny, int nz, std::vector<int64_t>& Ap, std::vector<int32_t>& Ai,
                           std::vector<double>& Ax, std::vector<double>& xyz) {
  const int n = nx * ny * nz;
  auto id = [&](int i, int j, int k) { return (k * ny + j) * nx + i; };
  Ap.assign(1, 0);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        std::vector<std::pair<int, double>> row;
        const int nb[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
        for (auto& d : nb) {
          const int a = i + d[0], b = j + d[1], c = k + d[2];
          if (a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) continue;
          row.push_back({id(a, b, c), -1.0});
        }
        row.push_back({id(i, j, k), (nz > 1 ? 6.0 : 4.0) + 0.01});
        std::sort(row.begin(), row.end());
        for (auto& e : row) {
          Ai.push_back(e.first);
          Ax.push_back(e.second);
        }
        Ap.push_back((int64_t)Ai.size());
        xyz.push_back(i);
        xyz.push_back(j);
        xyz.push_back(k);
      }
  (void)n;
}

// every (row, col) of B_s with row >= col is covered exactly once by the node's tiles
static bool covers(const Supernode& sn, const std::vector<Task>& tasks, bool forward, std::string& err) {
  const int ntot = sn.ncol + sn.nrow;
  std::vector<uint8_t> hit((size_t)ntot * sn.ncol, 0);
  for (const Task& t : tasks) {
    int r0 = 0, r1 = ntot, c0 = 0, c1 = sn.ncol;
    if (t.kind > 1) {
      if (forward) {
        r0 = t.r0, r1 = std::min(t.r0 + kFwdRows, ntot), c0 = t.c0, c1 = std::min(t.c0 + t.kind, sn.ncol);
        if (t.kind % 8 || t.kind > kFwdCols) { err = "forward tile width"; return false; }
      } else {
        r0 = t.r0, r1 = std::min(t.r0 + t.kind, ntot), c0 = t.c0, c1 = std::min(t.c0 + kBwdCols, sn.ncol);
        if (t.kind % 4 || t.kind > kBwdRows) { err = "backward tile height"; return false; }
      }
    } else if (t.kind == 1) {
      if (sn.ncol > kNarrowCols || sn.ld > kNodeMaxLd || (int64_t)sn.ld * sn.ncol * 4 > kNodeMaxBytes) {
        err = "node task too large";
        return false;
      }
    }
    for (int c = c0; c < c1; ++c)
      for (int r = std::max(r0, c); r < r1; ++r) ++hit[(size_t)r * sn.ncol + c];
  }
  for (int c = 0; c < sn.ncol; ++c)
    for (int r = c; r < ntot; ++r)
      if (hit[(size_t)r * sn.ncol + c] != 1) { err = "entry covered " + std::to_string(hit[(size_t)r * sn.ncol + c]) + " times"; return false; }
  return true;
}

struct Replay {
  std::vector<int64_t> seq;   // per task: order of execution (-1 never)
};

// the kernel's protocol: claim slots in order, wait for them to be filled, run,
// release (forward: pending of the parent; backward: done of the node), append
static bool replay(const Schedule& S, const PassSchedule& P, bool forward, int threads, int seed, Replay& out,
                   std::string& err) {
  const int nt = (int)P.tasks.size();
  const int nn = (int)(forward ? P.push.size() : P.push.size() / (1 + kPushKids));
  std::vector<std::atomic<int>> q(nt), pend(nn), done(nn);
  for (int i = 0; i < nt; ++i) q[i] = P.queue[i];
  for (int i = 0; i < nn; ++i) {
    pend[i] = forward ? P.pending[i] : 0;
    done[i] = 0;
  }
  std::atomic<int> c0{0}, c1{P.n_init}, stamp{0};
  std::atomic<bool> bad{false};
  out.seq.assign(nt, -1);
  std::vector<std::atomic<int>> runs(nt);
  for (auto& r : runs) r = 0;
  auto worker = [&](int w) {
    std::mt19937 rng(seed * 131 + w);
    int h = c0.fetch_add(1);
    for (;;) {
      if (h >= nt) return;
      int t;
      long spins = 0;
      while ((t = q[h].load(std::memory_order_acquire)) < 0) {
        if (++spins > 20000000L || bad) { bad = true; return; }
        std::this_thread::yield();
      }
      if (threads > 1 && rng() % 3 == 0) std::this_thread::sleep_for(std::chrono::microseconds(rng() % 20));
      runs[t]++;
      out.seq[t] = stamp.fetch_add(1);
      const Task& tk = P.tasks[t];
      const int hn = c0.fetch_add(1);
      if (forward) {
        const PushRec r = P.push[tk.node];
        if (r.x >= 0 && pend[r.x].fetch_sub(1) == 1) {
          const int base = c1.fetch_add(r.z);
          if (base + r.z > nt) { bad = true; return; }
          for (int i = 0; i < r.z; ++i) q[base + i].store(r.y + i, std::memory_order_release);
        }
      } else {
        const PushRec r = P.push[(size_t)tk.node * (1 + kPushKids)];
        if (r.z > 0 && (tk.kind <= 1 || done[tk.node].fetch_add(1) == r.w - 1)) {
          const int base = c1.fetch_add(r.z);
          if (base + r.z > nt) { bad = true; return; }
          for (int k = r.x; k < r.y; ++k) {
            const int j = k - r.x;
            const PushRec e = j < kPushKids ? P.push[(size_t)tk.node * (1 + kPushKids) + 1 + j] : P.kids[k];
            if (j < kPushKids && (e.x != P.kids[k].x || e.y != P.kids[k].y || e.z != P.kids[k].z)) { bad = true; return; }
            for (int i = 0; i < e.y; ++i) q[base + e.z + i].store(e.x + i, std::memory_order_release);
          }
        }
      }
      h = hn;
    }
  };
  std::vector<std::thread> th;
  for (int w = 0; w < threads; ++w) th.emplace_back(worker, w);
  for (auto& x : th) x.join();
  if (bad) { err = "stalled or overfilled queue"; return false; }
  for (int i = 0; i < nt; ++i)
    if (runs[i] != 1) { err = "task " + std::to_string(i) + " ran " + std::to_string(runs[i].load()) + " times"; return false; }
  (void)S;
  return true;
}

int main(int argc, char** argv) {
  (void)argc;
  (void)argv;
  struct Grid { int nx, ny, nz, leaf; };
  const Grid grids[] = {{18, 18, 18, 64}, {14, 16, 12, 32}, {70, 70, 1, 64}, {5, 4, 3, 8}};
  int checked = 0;
  for (const Grid& g : grids) {
    std::vector<int64_t> Ap;
    std::vector<int32_t> Ai;
    std::vector<double> Ax, xyz;
    grid_laplacian(g.nx, g.ny, g.nz, Ap, Ai, Ax, xyz);
    FactorInput in;
    in.nF = g.nx * g.ny * g.nz;
    in.Ap = Ap.data();
    in.Ai = Ai.data();
    in.Ax = Ax.data();
    in.coords = xyz.data();
    in.leaf_size = g.leaf;
    Factor f;
    std::string err;
    if (build_factor(in, f, err) != 0) return fail("factor: " + err);
    const auto& nd = f.nodes;
    const int nn = (int)nd.size();
    for (int s = 0; s < nn; ++s)
      if (nd[s].parent >= 0 && nd[s].parent <= s) return fail("nodes not children-first");
    std::map<int, int> by_col0;
    for (int s = 0; s < nn; ++s)
      if (nd[s].ncol > 0) by_col0[nd[s].col0] = s;
    const int narrows[] = {32, 64};
    const int bottoms[] = {0, 2, 3};
    const int heights[][2] = {{0, 0}, {1, 1}, {2, 1}, {3, 0}, {0, 3}, {8, 8}};
    const int tops[] = {0, 1, 3};
    for (int na : narrows)
      for (int nb : bottoms)
        for (auto& hh : heights)
          for (int top : tops) {
          if (nb > 0 && (hh[0] | hh[1]) && !(hh[0] == 2 && hh[1] == 1)) continue;
          if (top > 0 && !(na == 64 && (nb == 0 || nb == 2) && hh[0] == 2 && hh[1] == 1)) continue;
          if (top >= f.n_levels) continue;
          ScheduleOptions o;
          o.narrow_cols = na;
          o.bottom_levels = nb;
          o.subtree_height_f = hh[0];
          o.subtree_height_b = hh[1];
          o.top_levels = top;
          Schedule S;
          build_schedule(nd, f.n_levels, o, S);
          const std::string tag = "grid " + std::to_string(g.nx) + "x" + std::to_string(g.ny) + "x" +
                                  std::to_string(g.nz) + " narrow " + std::to_string(na) + " bottom " +
                                  std::to_string(nb) + " heights " + std::to_string(hh[0]) + "," +
                                  std::to_string(hh[1]) + " top " + std::to_string(top) + ": ";
          // the top levels have no tasks (their columns are solved between the passes)
          auto in_top = [&](int s) { return nd[s].level >= f.n_levels - top; };
          // level lists: tiles cover every block once, tasks sit on their node's level
          for (int pass = 0; pass < 2; ++pass) {
            const auto& L = pass == 0 ? S.fwd_levels : S.bwd_levels;
            const auto& off = pass == 0 ? S.fwd_off : S.bwd_off;
            if ((int)off.size() != f.n_levels + 1) return fail(tag + "level offsets");
            std::vector<std::vector<Task>> per(nn);
            for (int l = 0; l < f.n_levels; ++l)
              for (int64_t i = off[l]; i < off[l + 1]; ++i) {
                if (nd[L[i].node].level != l) return fail(tag + "task on the wrong level");
                per[L[i].node].push_back(L[i]);
              }
            for (int s = 0; s < nn; ++s) {
              if (nd[s].ncol == 0 || in_top(s)) {
                if (!per[s].empty()) return fail(tag + "tasks for an empty or top node");
                continue;
              }
              if (!covers(nd[s], per[s], pass == 0, err)) return fail(tag + (pass ? "backward " : "forward ") + err);
            }
          }
          // dynamic lists: each node of the levels >= nb once, merged subtrees whole
          for (int pass = 0; pass < 2; ++pass) {
            const PassSchedule& P = pass == 0 ? S.fwd : S.bwd;
            std::vector<int> seen(nn, 0), own(nn, 0);
            for (const Task& t : P.tasks) {
              if (t.kind != 0) {
                own[t.node]++;
                continue;
              }
              if (t.c0 < 1 || t.c0 > kSubtreeMaxNodes) return fail(tag + "merged subtree size");
              std::vector<int> mem;
              for (int i = 0; i < t.c0; ++i) {
                const auto it = by_col0.find(S.sub_nodes[t.r0 + i].col0);
                if (it == by_col0.end()) return fail(tag + "unknown merged node");
                mem.push_back(it->second);
              }
              if (mem.back() != t.node) return fail(tag + "merged subtree does not end at its root");
              for (size_t i = 0; i < mem.size(); ++i) {
                const int s = mem[i];
                seen[s]++;
                if (nd[s].ncol > kNarrowCols) return fail(tag + "merged node too wide");
                int a = s;   // s lies in the root's subtree
                while (a >= 0 && a != t.node) a = nd[a].parent;
                if (a != t.node) return fail(tag + "merged node outside its subtree");
                for (size_t j = 0; j < i; ++j)   // children first: no ancestor of s before it
                  for (int b = nd[s].parent; b >= 0; b = nd[b].parent)
                    if (b == mem[j]) return fail(tag + "merged subtree out of order");
              }
              for (int s = 0; s < nn; ++s) {   // every node of the subtree is a member
                if (nd[s].ncol == 0) continue;
                int a = s;
                while (a >= 0 && a != t.node) a = nd[a].parent;
                if (a == t.node && std::find(mem.begin(), mem.end(), s) == mem.end())
                  return fail(tag + "merged subtree incomplete");
              }
            }
            for (int s = 0; s < nn; ++s) {
              if (nd[s].ncol == 0) continue;
              if (in_top(s)) {
                if (seen[s] || own[s]) return fail(tag + "top node in the dynamic list");
                continue;
              }
              const bool dyn = nd[s].level >= S.bottom_used;
              if (seen[s] > 1 || (seen[s] && own[s])) return fail(tag + "node in the dynamic list twice");
              if (dyn != (seen[s] + (own[s] > 0) == 1)) return fail(tag + "node missing from the dynamic list");
              if (!dyn && own[s]) return fail(tag + "bottom-level node in the dynamic list");
            }
            // the forward pass's ready nodes are queued deepest first; a backward
            // completion releases the node with the tallest subtree first
            {
              std::vector<int> depth(nn, 0);
              for (int s = nn - 1; s >= 0; --s)
                if (nd[s].parent >= 0) depth[s] = depth[nd[s].parent] + 1;
              if (pass == 0)
                for (int i = 1; i < P.n_init; ++i)
                  if (depth[P.tasks[P.queue[i]].node] > depth[P.tasks[P.queue[i - 1]].node])
                    return fail(tag + "forward ready queue not deepest first");
              if (pass == 1)   // the nodes that wait on nothing start tallest first
                for (int i = 1; i < P.n_init; ++i)
                  if (nd[P.tasks[P.queue[i]].node].level > nd[P.tasks[P.queue[i - 1]].node].level)
                    return fail(tag + "backward start not tallest first");
              if (pass == 1)
                for (int s = 0; s < nn; ++s) {
                  const PushRec& r = P.push[(size_t)s * (1 + kPushKids)];
                  for (int k = r.x + 1; k < r.y; ++k)
                    if (nd[P.tasks[P.kids[k].x].node].level > nd[P.tasks[P.kids[k - 1].x].node].level)
                      return fail(tag + "backward release not tallest first");
                }
            }
            // replay the protocol; dependencies hold in the execution order
            for (int threads : {1, 24}) {
              Replay R;
              if (!replay(S, P, pass == 0, threads, checked, R, err)) return fail(tag + err);
              std::vector<int64_t> first(nn, INT64_MAX), last(nn, -1);
              for (size_t i = 0; i < P.tasks.size(); ++i) {
                const int s = P.tasks[i].node;
                first[s] = std::min(first[s], R.seq[i]);
                last[s] = std::max(last[s], R.seq[i]);
              }
              for (int s = 0; s < nn; ++s) {
                if (last[s] < 0) continue;
                for (int a = nd[s].parent; a >= 0; a = nd[a].parent) {
                  if (last[a] < 0) continue;
                  // forward: descendants finish before an ancestor starts; backward the reverse.
                  // With threads, "finish" is the claim order of the protocol's release, so the
                  // check uses the sequential replay only.
                  if (threads == 1 && pass == 0 && !(last[s] < first[a])) return fail(tag + "forward order");
                  if (threads == 1 && pass == 1 && !(last[a] < first[s])) return fail(tag + "backward order");
                }
              }
            }
          }
          ++checked;
          }
  }
  std::printf("ok %d schedules\n", checked);
  return 0;
}
