// Task lists and dependency records of the supernodal triangular solves (the
// W step's forward and backward passes, paper Sec. 4 "Efficient evaluation";
// Algorithm 1's W step).  Host-only C++ with no CUDA dependency, so the
// scheduling logic can be compiled and checked without a GPU; the device code
// reads the same structs.
#pragma once

#include <cstdint>
#include <vector>

#include "ffa_factor.h"

namespace ffa {

constexpr int kSolveThreads = 256;              // threads of a supernodal-solve block
constexpr int kSolveMinBlocks = 4;              // resident solve blocks per SM the registers allow
constexpr int kSolveWarps = kSolveThreads / 32;
constexpr int kFwdRows = 128;                   // forward wide task rows (4 per lane)
constexpr int kFwdCols = 32 * kSolveWarps;      // forward wide task: at most this many columns (W / warps per warp)
constexpr int kFwdBatch = 8;                    // forward: columns per lane in flight
constexpr int kBwdCols = 4 * kSolveWarps;       // backward wide task: output columns (4 per warp)
constexpr int kBwdRows = 1024;                  // backward wide task: at most this many rows
constexpr int kNarrowCols = 64;                 // node tasks: at most this many columns ...
constexpr int kNodeMaxLd = 4 * kSolveThreads;   // ... and at most one 4-row group per thread
constexpr int kNodeMaxBytes = 64 * 1024;        // ... and at most this much of B_s; taller narrow nodes
constexpr int kNarrowBwdRows = 256;             // are cut into 128-row (forward) / 256-row (backward) tiles
constexpr int kSubtreeMaxNodes = 16;            // dynamic passes: nodes of one merged bottom subtree
constexpr int kPushKids = 2;                    // backward push records: released nodes stored inline

struct NodeDev {
  int32_t col0, ncol, nrow, ld;   // ld: leading dimension of B_s (multiple of 4)
  int32_t l2_keep, pad;           // 1: stream B_s with the L2 keep-resident hint (the next pass reads it first)
  int64_t row_off, blk_off;
};

// kind 1: the whole node on one block; kind > 1: a wide task of B_node from
// (r0, c0) spanning kind columns (forward) or kind rows (backward); kind 0 (the
// dynamic passes only): a merged bottom subtree rooted at node, whose c0 nodes
// (node tasks, children before parents) start at entry r0 of the subtree node
// list and run in order on one block.  The node's descriptor travels with the
// task, so one 64-byte load brings both.
struct alignas(16) Task {
  int32_t node, r0, c0, kind;
  NodeDev nd;
};

// 16 bytes read as one vector by the device (layout of CUDA's int4)
struct alignas(16) PushRec {
  int32_t x, y, z, w;
};

// One pass (forward or backward) of the dynamic schedule.  Tasks of a node are
// contiguous in `tasks`.  push[s] says what a completed task of node s releases:
//   forward:  {p, first task of p, tasks of p, 0}, p = the node waiting on s or
//             -1; pending[p] counts the tasks of all nodes waiting on p, so the
//             task that brings it to zero makes p ready;
//   backward: {k0, k1, tasks of all nodes waiting on s, tasks of s} followed by
//             kPushKids inline copies of kids[k0], kids[k0 + 1] (stride
//             1 + kPushKids per node); the nodes waiting on s are kids[k0..k1) =
//             {first task, tasks, offset of its tasks among all of them, 0};
//             each waits on s alone, so the task that completes s (done[s]
//             reaches the task count) releases them all.
// queue holds the tasks that wait on nothing (n_init of them) followed by -1.
struct PassSchedule {
  std::vector<Task> tasks;
  std::vector<PushRec> push, kids;
  std::vector<int32_t> pending;   // forward only (per node)
  std::vector<int32_t> queue;
  int n_init = 0;
};

struct ScheduleOptions {
  int narrow_cols = kNarrowCols;   // node tasks: at most this many columns (<= kNarrowCols)
  int bottom_levels = 0;           // lowest levels run as one launch per level, outside the dynamic passes
  int subtree_height_f = 2;        // nb = 0: merged bottom subtrees of at most this height, forward pass
  int subtree_height_b = 1;        // ... backward pass (0: none)
  // L2 residency between passes: the forward pass reads the top levels last and
  // the backward pass reads them first (and the other way round for the bottom
  // levels and the next sweep's forward pass), so those blocks are streamed with
  // a keep-resident hint and all others with an evict-first hint
  int l2_keep_top = 2;             // forward: the top this-many levels with tasks (0: none)
  int l2_keep_bottom = 2;          // backward: levels below this one (0: none)
  int top_levels = 0;              // the top this-many levels have no tasks (their columns are
                                   // solved by the top-of-tree inverse between the passes)
};

struct Schedule {
  // level-synchronous lists: the tasks of level l are [off[l], off[l + 1])
  std::vector<Task> fwd_levels, bwd_levels;
  std::vector<int64_t> fwd_off, bwd_off;
  std::vector<NodeDev> sub_nodes;   // merged subtrees' nodes, both passes
  PassSchedule fwd, bwd;            // the dynamic passes over the levels >= bottom_used
  int bottom_used = 0;
};

// Builds both schedules for the supernodes of a factor (postorder: children
// before parents, `level` = height in the elimination tree).
void build_schedule(const std::vector<Supernode>& nodes, int n_levels, const ScheduleOptions& opt, Schedule& out);

}  // namespace ffa
