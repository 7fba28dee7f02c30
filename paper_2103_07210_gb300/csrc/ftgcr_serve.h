// Internal interface between the solver core (ftgcr.cu) and the request
// scheduler (ftgcr_server.cu): resumable persistent launches over a fixed
// table of solve slots.  A slot holds one running solve (a handle plus its
// right-hand side and solution pointers); each launch of the table runs every
// occupied slot for at most a given number of rounds and leaves the unfinished
// solves' complete state in device memory, so the next launch resumes them
// exactly where they stopped while newly begun solves join in free slots.  A
// solve's arithmetic depends only on its own handle (tiling, reduction order),
// never on the launch or on its neighbours, so its result is bitwise that of
// the same solve run alone.
#pragma once
#include <cuda_runtime.h>

#include "../../include/ftgcr.h"

namespace ftgcr {
namespace serve {

struct SlotTable;

// A table of max_slots (1..1024) slots for solves of one precision.
int table_create(int precision, int max_slots, SlotTable** out);
void table_destroy(SlotTable* t);

// Begin a solve of h in a free slot.  rhs, x: device pointers (x: initial
// guess in, solution out), valid until the solve has finished.  Enqueued on st;
// it may be enqueued behind a launch still in flight, and then joins the next.
// check: bit 0 rhs, bit 1 x are staged host inputs to test for non-finite
// values on the device first; a solve that fails the test does not start and
// finishes in the next launch with FTGCR_ERR_ARG.
int table_begin(SlotTable* t, int slot, ftgcr_handle* h, const double* rhs, double* x, const ftgcr_fault_plan* plan,
                cudaStream_t st, int check = 0);

// Run every occupied slot for at most max_rounds rounds (enqueued on st).
int table_run(SlotTable* t, int max_rounds, cudaStream_t st);

// Once st has passed table_run: finished[s] = 1 for every slot of that run
// whose solve ended in it (its handle then holds the result that ftgcr_stats()
// reports, and the slot is free again), else 0.  A launch whose grid barrier
// gave up ends every occupied slot, each with FTGCR_ERR_TIMEOUT.
int table_collect(SlotTable* t, cudaStream_t st, int* finished);

// Drop every occupied slot without results (after a failed launch).
void table_abandon(SlotTable* t, cudaStream_t st);

int table_occupied(const SlotTable* t);
int table_slots(const SlotTable* t);

// Device staging buffers of a handle for host right-hand sides and solutions.
double* handle_stage_rhs(ftgcr_handle* h);
double* handle_stage_x(ftgcr_handle* h);
long long handle_points(const ftgcr_handle* h);
int handle_precision(const ftgcr_handle* h);

}  // namespace serve
}  // namespace ftgcr
