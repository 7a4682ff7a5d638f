/*
 * kz_probe.h -- hardware probes used to state roofline denominators.
 *
 * The colour-index sweep (thesis Section 4.2 rules, bitset form) is bound by
 * integer logic throughput; no vendor figure for it is measured in the
 * environment, so the probe measures it on the device it runs on.  The
 * barrier probe exercises the failure path of the bounded grid barrier.
 */
#ifndef KZ_PROBE_H
#define KZ_PROBE_H

#include <stdint.h>

#include "kz.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Integer throughput probe (synchronous on `stream`).
 *   kind  0: 32-bit three-input logic ops (lop3.b32)
 *         1: 32-bit unsigned min (min.u32)
 *         2: three-input unsigned min (__vimin3_u32)
 *         3: one lop3.b32 feeding one min.u32 (2 operations per step)
 *         4: two lop3.b32 feeding one three-input min (3 operations per step)
 *   ops_per_s  receives the measured per-lane operations per second over the
 *              whole device (every SM busy, independent dependency chains);
 *              kinds 3 and 4 count every instruction of a step, so a rate
 *              above kind 0's shows the two instruction kinds issuing to
 *              different pipes
 *   ms         receives the measured kernel time
 * Returns KZ_ERR_ARG for a bad kind or null output, KZ_ERR_CUDA on failure.
 */
kz_status kz_probe_int_throughput(int32_t kind, double *ops_per_s, double *ms, void *stream);

/*
 * Failure-path probe of the bounded grid barrier (asynchronous on `stream`).
 * Runs the persistent sweep kernel on g with a barrier that waits for one
 * arrival more than the grid has, so every wait gives up after spin_limit
 * polls: the kernel records KZ_ERR_TIMEOUT in g's device status (read with
 * kz_fetch_stats) and returns, leaving the CUDA context usable.  The graph's
 * live state is not changed (no pass is applied).  Nothing here faults or
 * hangs the device; it exercises the path a lost CTA would take.
 */
kz_status kz_probe_barrier_timeout(kz_graph g, uint32_t spin_limit, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* KZ_PROBE_H */
