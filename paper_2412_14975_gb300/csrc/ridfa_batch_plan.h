// Host-side plan of one batched recognition (shared by ridfa_batch and ridfa_server): the
// chunking of every item, the reach tasks and their launch groups, the join segments, and the
// layout of the single device block the launches work in.  Not part of the public ABI.
//
// A device block starts with an image written on the host (plan_image: descriptors, zeroed
// counters, tickets and flags; image_bytes long) followed by device-only scratch (join partials,
// run lists, chunk maps, per-chunk summaries).  plan_enqueue launches the reach groups and the
// join on a stream; the accept bit of item i goes to d_accept[i].
#pragma once

#include <cuda_runtime_api.h>

#include <cstddef>
#include <cstdint>

#include "ridfa.h"

namespace ridfa {

struct BatchPlan;

BatchPlan *plan_new();
void plan_delete(BatchPlan *pl);

// Launch shape of the reach groups (the batch autotuner's knobs besides the chunk length).
struct BatchShape {
    uint32_t warps_cap = 0;   // warps per block at most (0: as many as the staging buffers allow)
    uint32_t set_mode = 0;    // tables too large to replicate: 0/1 a lane finishes all of its chunk's
                              // runs together (the set path), 2 one run per lane
};

// Plan items[0..n_items) over progs[0..n_progs) on `device` (the current device), items with
// n_chunks == 0 getting ceil(len / chunk_len) chunks.  Uploads program tables if needed.
// Errors: E_ARG, E_CHUNKS, E_UNSUPPORTED, E_NOMEM, E_CUDA.
int plan_build(BatchPlan *pl, const ridfa_program *const *progs, uint32_t n_progs,
               const ridfa_batch_item *items, uint32_t n_items, uint32_t chunk_len, int device,
               const BatchShape &shape = BatchShape{});

size_t plan_device_bytes(const BatchPlan *pl);   // whole device block
size_t plan_image_bytes(const BatchPlan *pl);    // leading part written from the host image
size_t plan_status_offset(const BatchPlan *pl);  // byte offset of the status word in the block

// Host image of the block for a block at device address `base` (pointers inside the
// descriptors depend on it); `img` holds plan_image_bytes bytes.
void plan_image(const BatchPlan *pl, uint8_t *base, uint8_t *img);

// Streams and events that let the reach groups of one batch (one per table layout) run
// concurrently: group 0 on the caller's stream, group g > 0 on aux[g - 1], joined back before the
// join launch.  Owned by the caller; created once with make_fork, released with free_fork.
constexpr int kMaxLaunchGroups = 5;
struct LaunchFork {
    cudaStream_t aux[kMaxLaunchGroups - 1] = {};
    cudaEvent_t ev[kMaxLaunchGroups] = {};
    bool ok = false;
};
int make_fork(LaunchFork *f);
void free_fork(LaunchFork *f);

// Enqueue the reach groups and the join on `st` for a block at `base` whose image is in place.
// zero_counters: clear the task tickets and status word first (graph replays).  fork: run the
// reach groups concurrently (null: one after another on `st`).
int plan_enqueue(const BatchPlan *pl, uint8_t *base, uint8_t *d_accept, cudaStream_t st, bool zero_counters,
                 const LaunchFork *fork = nullptr);

struct PlanStats {
    uint64_t total_bytes, total_chunks;
    uint32_t n_programs, n_launches, n_tasks, n_segments;
};
PlanStats plan_stats(const BatchPlan *pl);

}  // namespace ridfa
