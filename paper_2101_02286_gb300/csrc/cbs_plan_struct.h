// cbs_plan_struct.h -- the opaque plan and batch objects of the C-ABI
// (shared by the translation units that implement entry points).
#pragma once
#include <string>
#include <vector>

#include "cbs_closure.cuh"
#include "cbs_internal.h"
#include "cbs_line.cuh"
#include "cbs_long.cuh"
#include "cbs_var.cuh"

using cbs::DevLineTables;
using cbs::LineArgs;
using cbs::LineTables;
using cbs::LongArgs;
using cbs::LongGeom;
using cbs::LongWarpArgs;
using cbs::LwIface;
using cbs::VarArgs;

struct cbs_batch {
  std::vector<cbs_plan*> plans;
  void* dprobs = nullptr;
  void* ditems = nullptr;
  int nitems = 0, count = 0, grid = 1;
  size_t smem = 0;
  int64_t unknowns = 0;
  int mode = 0;                   // cbs_batch_set_mode
  bool persistent = true;         // every problem fits the persistent launch
  std::string why;                // else: the first problem that does not, and why
  int device = -1;                // device current at creation
  std::vector<int> order_fp64;    // per-problem launches: FP64 problems, largest first
  std::vector<int> order_other;   // the others, largest first
  cudaStream_t side = nullptr;    // per-problem launches: the FP64 problems' stream
  cudaEvent_t fork = nullptr, join = nullptr;
};

struct cbs_plan {
  cbs_desc desc;
  int n = 0, r = 1, kind = 0, M = 16, ks = 0;
  int variant = 0;     // cbs_plan_set_variant: 0 automatic (TMA kernel where it qualifies), 1 line kernels
  int tile_lines = 0;  // TMA kernel: lines per tile (0: the default of the direction)
  int fault = 0;       // cbs_plan_inject_fault (test of the timeout path)
  int64_t nlines = 0;
  LineTables host;
  DevLineTables dev;
  void* dbuf = nullptr;
  int* dstatus = nullptr;
  LineArgs args;
  bool var = false;
  VarArgs vargs;
  // long lines (kind 1): segments across CTAs
  LineTables inner, inner_small;      // segment-level tables (the second for msmall-row segments)
  DevLineTables dev_inner, dev_inner_small;
  bool inner_full = false;            // every segment's bulk is a whole number of 16-row partitions
  LongArgs largs;
  LongGeom lgeom;
  void* lbuf = nullptr;
  void* lbuf_small = nullptr;
  void* sbuf = nullptr;
  int inner_threads = 0;
  bool long_warp = false;             // x-lines, a warp per segment (decoupled outer system)
  cbs::LongWarpArgs lwargs;
  cbs::LwIface lwifc[2];              // compact inner systems: 32 and 31 partitions
  void* lwbuf = nullptr;              // their device tables
  // one-sided boundary closures (acyclic derivatives): the correction launch
  bool closure = false;
  cbs::ClosureArgs cargs;
  void* cbuf = nullptr;
};

namespace cbs {
// Record the calling thread's last error (cbs_last_error_string) and the
// launch count of the last solve; return `s`.
cbs_status set_error(cbs_status s, const std::string& msg);
void set_launch_count(int n);
// inner_small: tables of the msmall-row segments (whole-16-row layout), or
// null when every segment uses `inner`.
bool long_warp_fits(int R, int K, int in_size, bool yz);
cudaError_t launch_long_warp(int mode, int R, bool in64, bool out64, const LongArgs& a, const DevLineTables& inner,
                             const DevLineTables* inner_small, const LongWarpArgs& wa, const LwIface* ifc,
                             cudaStream_t s, int* launches);
cudaError_t launch_long(int mode, int R, bool in64, bool out64, const LongArgs& a, const LongGeom& gm,
                        const DevLineTables& outer,
                        const DevLineTables& inner, const DevLineTables* inner_small, bool full, cudaStream_t s,
                        int* launches);
}  // namespace cbs
