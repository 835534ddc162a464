/*
 * psfsim testing hooks: entry points that exist so that tests can drive the
 * library's failure paths on a GPU without faulting, trapping or hanging it.
 * They are not part of the method (the paper has no counterpart) and a
 * production caller has no reason to use them.
 */
#ifndef PSFSIM_TESTING_H
#define PSFSIM_TESTING_H

#include <stddef.h>
#include <stdint.h>

#include "psfsim.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The tensor-core forward of psfsim_forward (SPLIT_BF16 or BF16 plan, B <= 80
 * scenes; or FUSED plan, B <= 64 scenes; same scratch as psfsim_forward) run
 * on ONE CTA with every device-side wait bounded by wait_ns nanoseconds
 * (1 us .. 2 s), and with the shared-memory load number stall_load (counted
 * from 0 in the CTA's issue order: for FUSED, the x tile of the CTA's k-tile
 * number stall_load; -1: none) never issued: the MMA issuer's wait for that
 * stage then runs out, the kernel records PSFSIM_ERR_TIMEOUT in the plan's
 * status word, every role leaves its loop, waits (bounded) for the copies and
 * MMAs it already issued, releases its tensor memory and returns.  Images are
 * then incomplete.  Nothing is left in flight and the context stays usable:
 * psfsim_reset_status and a normal psfsim_forward work right after.
 * PSFSIM_ERR_ARG for out-of-range limits or batches, PSFSIM_ERR_UNSUPPORTED
 * for other storages. */
int psfsim_debug_forward_stall(psfsim_t h, const float *d_x, int B, float *d_y, void *d_scratch,
                               size_t scratch_bytes, uint64_t wait_ns, int64_t stall_load, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PSFSIM_TESTING_H */
