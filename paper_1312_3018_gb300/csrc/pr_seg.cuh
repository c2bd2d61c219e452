// Segmented pull PageRank (pr_seg.cu): the plan of a partitioned graph and one iteration's
// compute phase, for FP32 and FP16-stored contributions. pagerank.cu runs the iteration
// loop (publish, compute, finalize) and calls in here for the compute phase.
#pragma once

#include "common.cuh"

namespace gg {

struct SegWs;

// Layout parameters of a plan (0 picks the default).
struct SegParams {
  int log2;   // source-segment size 2^log2 (6 ... 15)
  int chunk;  // entries per phase-1 chunk (64 ... kSegChunkMax)
  int bin;    // partial sums per phase-2 bin (64 ... 28672)
};

// Per-iteration arguments. Index p is the partition.
struct SegIter {
  const void* x[2];       // contributions of this iteration
  const void* ghost[2];   // ghost-slot contributions (published this iteration)
  void* xn[2];            // contributions of the next iteration
  void* r[2];             // ranks (FP32)
  const double* scal;     // device scalars; the FP32 constant term is a float at scal + 4
  double* slots;          // FP64 residual slots
  uint32_t nslots;
  float d;                // damping
  float d_over_n;         // damping / n (scaled FP16 sums)
  float n;                // n (scaled FP16 contributions)
  bool fp16;              // contributions stored as FP16 scaled by n
};

// Builds (or keeps) the plan of g's current partition with the given parameters. Returns
// GRAPH_OK with *usable = false when the graph exceeds a limit of the segmented layout
// (then the caller uses the per-edge gather kernel); errors (ENOMEM, ECUDA) free the plan.
graph_status seg_prepare(graph* g, const SegParams& prm, bool* usable);

// Launches one iteration's compute (phase 1, phase 2, degree-zero vertices) on g->stream.
graph_status seg_launch(graph* g, const SegIter& it);

// Kernel launches per iteration.
int seg_launches_per_iter(const graph* g);

void free_seg(graph* g);

}  // namespace gg
