// Task lists and dependency records of the supernodal triangular solves; see
// ffa_schedule.h.
#include "ffa_schedule.h"

#include <algorithm>

namespace ffa {

namespace {

// Tasks of one dynamic pass: the tasks of the levels >= nb taken from the level
// lists, with each maximal bottom subtree of height <= H whose nodes are all
// node tasks (at most kSubtreeMaxNodes of them) replaced by one task of kind 0
// that runs the subtree's nodes in order on one block.
std::vector<Task> dynamic_list(const std::vector<Supernode>& nd, const std::vector<NodeDev>& nodes,
                               const std::vector<char>& all_node_tasks, const std::vector<int32_t>& size,
                               const std::vector<Task>& all, const std::vector<int64_t>& off, int nb, int H,
                               const std::vector<char>& keep, std::vector<NodeDev>& sub_nodes) {
  const int nn = (int)nd.size();
  if (nb > 0) H = 0;
  auto mergeable = [&](int s) {
    return nd[s].ncol > 0 && nd[s].level <= H && all_node_tasks[s] && size[s] <= kSubtreeMaxNodes;
  };
  std::vector<int32_t> root(nn, -1);
  for (int s = 0; s < nn; ++s) {
    if (H <= 0 || !mergeable(s)) continue;
    int r = s;
    while (nd[r].parent >= 0 && mergeable(nd[r].parent)) r = nd[r].parent;
    root[s] = r;
  }
  // members of each merged subtree in increasing node order (children have
  // smaller indices than their parents, so that order runs children first)
  std::vector<std::vector<int32_t>> members(nn);
  for (int s = 0; s < nn; ++s)
    if (root[s] >= 0 && nd[s].ncol > 0) members[root[s]].push_back(s);
  std::vector<int32_t> first(nn, 0), count(nn, 0);
  for (int r = 0; r < nn; ++r) {
    if (members[r].empty()) continue;
    first[r] = (int32_t)sub_nodes.size();
    count[r] = (int32_t)members[r].size();
    for (int m : members[r]) {
      sub_nodes.push_back(nodes[m]);
      sub_nodes.back().l2_keep = keep[m];
    }
  }
  std::vector<Task> out;
  for (int64_t i = off[nb]; i < (int64_t)all.size(); ++i) {
    const int s = all[i].node;
    const int r = root[s];
    if (r < 0) out.push_back(all[i]);
    else if (r == s) out.push_back(Task{s, first[s], count[s], 0, nodes[s]});
    else continue;
    out.back().nd.l2_keep = keep[s];
  }
  return out;
}

// per-node task ranges of a list (a node's tasks are contiguous)
void ranges(const std::vector<Task>& all, int nn, std::vector<int32_t>& t0, std::vector<int32_t>& cnt) {
  t0.assign(nn, 0);
  cnt.assign(nn, 0);
  for (size_t i = 0; i < all.size(); ++i) {
    const int s = all[i].node;
    if (cnt[s]++ == 0) t0[s] = (int32_t)i;
  }
}

// nearest ancestor with tasks in a pass's list
std::vector<int32_t> nearest(const std::vector<Supernode>& nd, const std::vector<int32_t>& cnt) {
  const int nn = (int)nd.size();
  std::vector<int32_t> up(nn, -1);
  for (int s = 0; s < nn; ++s) {
    int p = nd[s].parent;
    while (p >= 0 && cnt[p] == 0) p = nd[p].parent;
    up[s] = p;
  }
  return up;
}

}  // namespace

void build_schedule(const std::vector<Supernode>& nd, int n_levels, const ScheduleOptions& opt, Schedule& out) {
  const int nl = n_levels;
  const int nn = (int)nd.size();
  const int narrow = std::min(opt.narrow_cols, kNarrowCols);
  auto is_node_task = [&](const Supernode& sn) {
    return sn.ncol <= narrow && sn.ld <= kNodeMaxLd && (int64_t)sn.ld * sn.ncol * 4 <= kNodeMaxBytes;
  };
  std::vector<NodeDev> nodes(nn);
  std::vector<std::vector<Task>> fl(nl), bl(nl);
  for (int s = 0; s < nn; ++s) {
    const Supernode& sn = nd[s];
    nodes[s] = NodeDev{sn.col0, sn.ncol, sn.nrow, sn.ld, 0, 0, sn.row_off, sn.blk_off};
    const int ntot = sn.ncol + sn.nrow;
    if (sn.ncol == 0 || sn.level >= nl - opt.top_levels) continue;
    if (is_node_task(sn)) {
      fl[sn.level].push_back(Task{s, 0, 0, 1, nodes[s]});
      bl[sn.level].push_back(Task{s, 0, 0, 1, nodes[s]});
      continue;
    }
    // a narrow node too tall for one block is cut into row tiles that each
    // stream a few load rounds (its tasks sit on the critical path of the
    // middle levels); wider nodes take the full tile shapes (smaller wide
    // tasks on the narrow top levels were measured slower: the fixed cost of
    // a task outweighs the shorter tail)
    const bool narrow_node = sn.ncol <= narrow;
    const int wf = narrow_node ? (sn.ncol + 7) / 8 * 8 : kFwdCols;
    const int wb = narrow_node ? kNarrowBwdRows : kBwdRows;
    for (int r0 = 0; r0 < ntot; r0 += kFwdRows)
      for (int c0 = 0; c0 < sn.ncol; c0 += wf) {
        const int rmax = std::min(r0 + kFwdRows, ntot) - 1;
        if (rmax < c0) continue;  // entirely above the diagonal of inv(L_ss)
        fl[sn.level].push_back(Task{s, r0, c0, wf, nodes[s]});
      }
    for (int c0 = 0; c0 < sn.ncol; c0 += kBwdCols)
      for (int r0 = 0; r0 < ntot; r0 += wb) {
        const int rmax = std::min(r0 + wb, ntot) - 1;
        if (rmax < c0) continue;
        bl[sn.level].push_back(Task{s, r0, c0, wb, nodes[s]});
      }
  }
  out = Schedule{};
  out.fwd_off.assign(1, 0);
  out.bwd_off.assign(1, 0);
  for (int l = 0; l < nl; ++l) {
    out.fwd_levels.insert(out.fwd_levels.end(), fl[l].begin(), fl[l].end());
    out.bwd_levels.insert(out.bwd_levels.end(), bl[l].begin(), bl[l].end());
    out.fwd_off.push_back((int64_t)out.fwd_levels.size());
    out.bwd_off.push_back((int64_t)out.bwd_levels.size());
  }

  // The dynamic passes cover the nodes on levels >= nb (closed under
  // ancestors); the levels below run as one launch each, before the forward
  // dynamic launch and after the backward one.
  const int nb = std::min(opt.bottom_levels, nl);
  out.bottom_used = nb;
  std::vector<char> all_node_tasks(nn, 1);   // every node of the subtree is a node task (or empty)
  std::vector<int32_t> size(nn, 0);          // nodes with columns in the subtree
  for (int s = 0; s < nn; ++s) {             // postorder: children first
    const Supernode& sn = nd[s];
    // a merged subtree holds no node of the top levels (they have no tasks)
    all_node_tasks[s] = all_node_tasks[s] && (sn.ncol == 0 || is_node_task(sn)) && sn.level < nl - opt.top_levels;
    size[s] += sn.ncol > 0 ? 1 : 0;
    if (sn.parent >= 0) {
      all_node_tasks[sn.parent] = all_node_tasks[sn.parent] && all_node_tasks[s];
      size[sn.parent] += size[s];
    }
  }
  std::vector<char> keep_f(nn, 0), keep_b(nn, 0);
  for (int s = 0; s < nn; ++s) {
    keep_f[s] = nd[s].level >= nl - opt.top_levels - opt.l2_keep_top;
    keep_b[s] = nd[s].level < opt.l2_keep_bottom;
  }
  out.fwd.tasks = dynamic_list(nd, nodes, all_node_tasks, size, out.fwd_levels, out.fwd_off, nb, opt.subtree_height_f,
                               keep_f, out.sub_nodes);
  out.bwd.tasks = dynamic_list(nd, nodes, all_node_tasks, size, out.bwd_levels, out.bwd_off, nb, opt.subtree_height_b,
                               keep_b, out.sub_nodes);
  // the two lists merge different subtrees, so a node can have tasks in one
  // pass only: each pass has its own dependencies
  std::vector<int32_t> t0f, ntf, t0b, ntb;
  ranges(out.fwd.tasks, nn, t0f, ntf);
  ranges(out.bwd.tasks, nn, t0b, ntb);
  const std::vector<int32_t> up_f = nearest(nd, ntf), up_b = nearest(nd, ntb);

  // forward: s waits on the tasks of the nodes whose nearest ancestor with tasks is s
  PassSchedule& F = out.fwd;
  F.push.assign(nn, PushRec{-1, 0, 0, 0});
  F.pending.assign(nn, 0);
  for (int s = 0; s < nn; ++s)
    if (ntf[s] > 0 && up_f[s] >= 0) {
      const int p = up_f[s];
      F.push[s] = PushRec{p, t0f[p], ntf[p], 0};
      F.pending[p] += ntf[s];
    }
  // the ready nodes enter the queue deepest first (the distance to the root is
  // the length of the chain each one starts), ties in node order
  std::vector<int32_t> depth(nn, 0);
  for (int s = nn - 1; s >= 0; --s)   // parents after children: walk down from the roots
    if (nd[s].parent >= 0) depth[s] = depth[nd[s].parent] + 1;
  std::vector<int32_t> ready;
  for (int s = 0; s < nn; ++s)
    if (ntf[s] > 0 && F.pending[s] == 0) ready.push_back(s);
  std::stable_sort(ready.begin(), ready.end(), [&](int a, int b) { return depth[a] > depth[b]; });
  for (int s : ready)
    for (int i = 0; i < ntf[s]; ++i) F.queue.push_back(t0f[s] + i);
  F.n_init = (int)F.queue.size();
  F.queue.resize(F.tasks.size(), -1);

  // backward: s waits on its nearest ancestor with tasks alone
  PassSchedule& B = out.bwd;
  std::vector<std::vector<int32_t>> kids(nn);
  for (int s = 0; s < nn; ++s)
    if (ntb[s] > 0 && up_b[s] >= 0) kids[up_b[s]].push_back(s);
  // a completion releases the node with the tallest subtree first: its chain to
  // the leaves is the longest
  for (auto& k : kids) std::stable_sort(k.begin(), k.end(), [&](int a, int b) { return nd[a].level > nd[b].level; });
  B.push.assign((size_t)nn * (1 + kPushKids), PushRec{0, 0, 0, 0});
  for (int s = 0; s < nn; ++s) {
    const int k0 = (int)B.kids.size();
    int total = 0;
    for (int c : kids[s]) {
      B.kids.push_back(PushRec{t0b[c], ntb[c], total, 0});
      total += ntb[c];
    }
    const int k1 = (int)B.kids.size();
    B.push[(size_t)s * (1 + kPushKids)] = PushRec{k0, k1, total, ntb[s]};
    for (int j = 0; j < kPushKids && k0 + j < k1; ++j) B.push[(size_t)s * (1 + kPushKids) + 1 + j] = B.kids[k0 + j];
  }
  // the nodes that wait on nothing (the root, or the nodes below the top levels
  // without tasks) start tallest subtree first
  std::vector<int32_t> roots;
  for (int s = nn - 1; s >= 0; --s)
    if (ntb[s] > 0 && up_b[s] < 0) roots.push_back(s);
  std::stable_sort(roots.begin(), roots.end(), [&](int a, int b) { return nd[a].level > nd[b].level; });
  for (int s : roots)
    for (int i = 0; i < ntb[s]; ++i) B.queue.push_back(t0b[s] + i);
  B.n_init = (int)B.queue.size();
  B.queue.resize(B.tasks.size(), -1);
}

}  // namespace ffa
