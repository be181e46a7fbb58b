/*
 * tc_debug.h -- failure-path test hooks of libtc (see tc.h).
 *
 * The paper has no counterpart: these calls exist so that tests can drive
 * the library's error paths without faulting or hanging a GPU.  They change
 * process-wide (allocation failures) or per-device (waits) state and are not
 * meant for production use; tc_debug_reset() undoes all of them.
 */
#ifndef TC_DEBUG_H
#define TC_DEBUG_H

#include <stdint.h>

#include "tc.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Bounded device waits, made to run out.  The preprocessing kernels wait
 * (spin) on status words that earlier tiles of the same launch publish
 * (decoupled look-back); every such wait gives up after a bounded number of
 * iterations, records the failure in the call's error word, and the call
 * returns TC_ERR_TIMEOUT with nothing computed from incomplete data (later
 * kernels of the call return at entry).  On the CURRENT device:
 *   spin_limit        iterations before a wait gives up (default 2^24)
 *   unpublished_tile  >= 0: the radix-sort tile with this number never
 *                     publishes its status, so the tiles after it wait on a
 *                     word that nothing sets and give up after spin_limit
 *                     iterations; < 0: every tile publishes (default)
 * Synchronises the device.  Returns TC_ERR_CUDA if the device rejects it.
 */
tc_status tc_debug_set_wait_limit(uint32_t spin_limit, int32_t unpublished_tile);

/*
 * Allocation failures, injected on the host: of the library's next device
 * allocations (workspaces, engine buffers, host-call staging), the first
 * `skip` succeed and the `count` after them fail as if the device were out
 * of memory (the call returns TC_ERR_OOM and releases what it had taken).
 * count <= 0 turns injection off.  Process-wide.
 */
tc_status tc_debug_fail_allocations(int32_t skip, int32_t count);

/* Default wait limit and no unpublished tile on the current device, and no
 * injected allocation failures. */
tc_status tc_debug_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* TC_DEBUG_H */
