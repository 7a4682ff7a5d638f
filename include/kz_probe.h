/*
 * kz_probe.h -- hardware probes used to state roofline denominators.
 *
 * The colour-index sweep (thesis Section 4.2 rules, bitset form) is bound by
 * integer logic throughput, for which no vendor figure is measured in the
 * environment; these probes measure it on the device they run on.
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
 *   ops_per_s  receives the measured per-lane operations per second over the
 *              whole device (every SM busy, independent dependency chains)
 *   ms         receives the measured kernel time
 * Returns KZ_ERR_ARG for a bad kind or null output, KZ_ERR_CUDA on failure.
 */
kz_status kz_probe_int_throughput(int32_t kind, double *ops_per_s, double *ms, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* KZ_PROBE_H */
