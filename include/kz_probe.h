/*
 * kz_probe.h -- hardware probes used to state roofline denominators.
 *
 * The colour-index sweep (thesis Section 4.2 rules, bitset form) is bound by
 * integer logic throughput, and its tensor-core form by the fp8 MMA rate;
 * no vendor figure for either is measured in the environment, so these
 * probes measure them on the device they run on.
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
 * tcgen05 fp8 MMA throughput probe (synchronous on `stream`): one CTA per SM
 * (or two, ctas_per_sm = 2) issues MMAs of M = 128, N = n (128 or 256),
 * K = 32, E4M3 operands from shared memory, fp32 accumulation in tensor
 * memory, back to back, and waits for them.  The operand layout in shared
 * memory is
 *   layout 0: no swizzle, K halves rows x 16 bytes apart (the layout one TMA
 *             box of the tensor path's byte matrix produces);
 *   layout 1: no swizzle, K halves 128 bytes apart, 8-row groups 256 apart;
 *   layout 2: 128-byte swizzle, K-major, one 128-byte row per operand row.
 *   flops_per_s  receives 2 x M x N x K x MMAs / time over the whole device
 *   ms           receives the measured kernel time
 * Returns KZ_ERR_ARG for a bad argument or null output, KZ_ERR_TIMEOUT if
 * the bounded wait for the MMAs gave up, KZ_ERR_CUDA on failure.
 */
kz_status kz_probe_mma_throughput(int32_t layout, int32_t n, int32_t ctas_per_sm, double *flops_per_s, double *ms,
                                  void *stream);

/*
 * TMA load throughput probe (synchronous on `stream`): one thread per CTA,
 * one CTA per SM (or two, ctas_per_sm = 2), streams 16 KB stages from an
 * L2-resident 32 MB buffer into a six-stage shared-memory ring, re-issuing a
 * stage as soon as its previous load has landed.
 *   mode 0: tensor map of 8-byte elements, box 256 x 2 (4 KB as two
 *           contiguous 2 KB runs: the tensor path's operand box)
 *   mode 1: tensor map of bytes, box 128 x 32 rows, 128-byte swizzle
 *   mode 2: untiled bulk copies of 4 KB
 *   mode 3: tensor map of 8-byte elements, box 256 x 8 (16 KB)
 *   bytes_per_s  receives the bytes landed per second over the device
 *   ms           receives the measured kernel time
 * Returns KZ_ERR_ARG for a bad argument or null output, KZ_ERR_UNSUPPORTED
 * without a tensor-map encoder, KZ_ERR_TIMEOUT if a bounded wait gave up,
 * KZ_ERR_CUDA on failure.
 */
kz_status kz_probe_tma_throughput(int32_t mode, int32_t ctas_per_sm, double *bytes_per_s, double *ms, void *stream);

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
