// Stepwise query objects driven by the query server (serve.cu). Each owns its workspace,
// its counters and a non-blocking stream, shares the graph's partitions read-only, and
// advances one BSP superstep at a time without blocking the host: the server issues a
// step, later finds its event complete, reads the step's counters and issues the next.
// None of these functions allocates except *_create.
#pragma once

#include "common.cuh"

namespace gg {

// ---- SSSP: one query per job (sssp.cu) ------------------------------------------------
struct SsspJob;
size_t sssp_job_bytes(const graph* g);  // device bytes one job holds
graph_status sssp_job_create(graph* g, SsspJob** out);
void sssp_job_destroy(graph* g, SsspJob* j);
// Starts a search from source; the distances go to dst (n uint32, global order; host
// memory should be pinned) when the job finishes. delta: near-far bucket width (0: plain
// active-set rounds).
graph_status sssp_job_start(graph* g, SsspJob* j, uint32_t source, uint32_t* dst,
                            int dst_mem, uint32_t delta);
// Non-blocking: 0 while running, 1 once dst holds the result, < 0 a graph_status error
// (the job is then idle). *rounds receives the supersteps run so far.
int sssp_job_poll(graph* g, SsspJob* j, int* rounds);

// ---- SSSP: up to sb_job_lanes() queries sharing one batched search (ssspb.cu) ---------
struct SbJob;
uint32_t sb_job_lanes();
size_t sb_job_bytes(const graph* g);  // device bytes one batched job holds
graph_status sb_job_create(graph* g, SbJob** out);
void sb_job_destroy(graph* g, SbJob* j);
// Starts k searches; search l's distances go to dst[l] when the job ends. delta: near-far
// bucket width shared by the lanes (0: plain rounds).
graph_status sb_job_start(graph* g, SbJob* j, const uint32_t* sources, uint32_t k,
                          uint32_t* const* dst, int dst_mem, uint32_t delta);
// As sssp_job_poll, for all k searches at once.
int sb_job_poll(graph* g, SbJob* j, int* rounds);

// ---- BFS: up to 64 queries as bit lanes of one multi-source search (msbfs.cu) ----------
struct BfsLanes;
size_t bfs_lanes_bytes(const graph* g, uint32_t nlanes);
graph_status bfs_lanes_create(graph* g, uint32_t nlanes, BfsLanes** out);
void bfs_lanes_destroy(graph* g, BfsLanes* b);
// Lanes that hold no search.
uint64_t bfs_lanes_free(const BfsLanes* b);
bool bfs_lanes_busy(const BfsLanes* b);  // a superstep is in flight
// Joins a search from source on a free lane at the next superstep boundary (only while no
// superstep is in flight); its levels go to dst (n uint32) when the lane finishes.
graph_status bfs_lanes_admit(BfsLanes* b, int lane, uint32_t source, uint32_t* dst,
                             int dst_mem);
// Issues the next superstep for every lane holding a search (no-op if none).
graph_status bfs_lanes_launch(graph* g, BfsLanes* b);
// Non-blocking: once the superstep in flight has completed, reads its counters, and for
// every lane that gained no vertex (its search is over) writes the levels to the lane's
// dst, frees the lane, records done_ev after those writes, and sets *finished (the lanes)
// and steps[lane] (the lane's supersteps). Returns 1 if a superstep completed, else 0, or
// a graph_status error.
int bfs_lanes_poll(graph* g, BfsLanes* b, uint64_t* finished, int* steps,
                   cudaEvent_t done_ev);

}  // namespace gg
