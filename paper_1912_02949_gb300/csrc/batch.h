// Batched engine of libscgal: many small FP32 MaxCut solves advanced by
// persistent launches (k_batch.cu), driven by the serving loop (server.cu).
#pragma once

#include "internal.h"

namespace scgal {

// batched engine (FP32 MaxCut instances small enough for one block)
struct BatchStatus {        // what a batched launch left of one instance
    long long t, conv_t;
    int converged, err;
};
bool batch_eligible(const scgal_ctx* h);
const void* handle_params(const scgal_ctx* h);   // the handle's KP<float> (host copy)
size_t batch_slot_bytes();                       // size of one batched-engine slot descriptor
// Builds the instance's sliced graph layout (device memory owned by the handle)
// and writes its slot descriptor (batch_slot_bytes() bytes) to out.
int batch_prepare(scgal_ctx* h, void* out);
// One persistent launch over the slots d_active[0 .. nact): each instance runs
// until it converges, reaches T_max, has run `iters` iterations or (after its
// first iteration) the launch has run for budget_ns; d_status[slot] is written.
int batch_variant(const void* desc);             // kernel variant of a slot descriptor, < BATCH_NVAR
constexpr int BATCH_NVAR = 12;                   // 6 one-block variants, 6 clustered
constexpr int BATCH_CTL_DEADLINE = 24;           // int offset of the deadline in the control block
constexpr int BATCH_CTL_INTS = 32;               // ints of the control block
struct BatchLaunch;                              // per-variant streams and events of the launches
BatchLaunch* batch_launch_create();
void batch_launch_destroy(BatchLaunch* L);
// One round: the slots d_active[0 .. sum counts), grouped by variant in variant
// order (counts[v] of variant v), one persistent launch per variant, all after
// the work already on stream s and before the work enqueued on it next.  Each
// instance runs until it converges, reaches T_max, has run `iters` iterations
// or (after its first iteration) the round has run for budget_ns;
// d_status[slot] is written.  d_ctl: BATCH_CTL_INTS ints of device scratch.
int launch_batch(BatchLaunch* L, const void* d_slots, const int* d_active, const int* counts, int* d_ctl, int iters,
                 unsigned long long budget_ns, BatchStatus* d_status, cudaStream_t s);
// The host's view of the handle from a status; *done when it converged or
// reached T_max (then *out holds its last iteration record).
int batch_apply(scgal_ctx* h, const BatchStatus& st, scgal_stats* out, int* done);

}  // namespace scgal
