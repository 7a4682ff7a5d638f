/*
 * kz_learned.h -- the learned schedule of the colour-index kernelization.
 *
 * The thesis (Section 4.2) gives the two colour-index rules and nothing about
 * the order in which elements are tested.  Because the greatest fixpoint of
 * monotone deletion rules is unique, any order that deletes only failing
 * elements and ends with a sweep that deletes nothing reaches the same
 * kernel.  This interface adds a small network that ranks edges by how likely
 * they are to fail, so that a sweep can test the likely failures first.
 *
 * Network: 16 features -> 64 -> 64 -> 1, ReLU hidden layers, logistic output.
 * Inference uses bf16 weights with fp32 accumulation; training keeps fp32
 * master weights (Adam).  Weights are one flat float array of
 * KZ_MLP_PARAMS values in the order W1[64][16], b1[64], W2[64][64], b2[64],
 * w3[64], b3.
 *
 * Features of an edge {u, v} (all from per-vertex statistics of the live
 * graph, computed once per round):
 *   0,1  live degree of u, v divided by n
 *   2,3  vertex colour-cover slack of u, v: (classes covered - (k-1)) / k
 *   4,5  smallest per-class neighbour count of u, v divided by n / k
 *   6,7  relative live-degree change of u, v since the previous round
 *   8    k / 64          9  round index / 32        10  live edge density
 *   11   min(deg u, deg v) / max(deg u, deg v)     12  (deg u + deg v) / (2 n)
 *   13   log2(n) / 16    14  fraction of live vertices
 *   15   1 - exp(-lambda), lambda = sum over the classes c other than the
 *        endpoints' of exp(-cnt_u[c] cnt_v[c] / |C_c|), cnt_u[c] the live
 *        neighbours of u in class c: the chance that a needed class holds no
 *        common neighbour if the endpoints' neighbours in each class were
 *        random (a scale-free summary of the per-class degrees)
 */
#ifndef KZ_LEARNED_H
#define KZ_LEARNED_H

#include <stdint.h>

#include "kz.h"

#ifdef __cplusplus
extern "C" {
#endif

#define KZ_MLP_FEATURES 16
#define KZ_MLP_HIDDEN 64
#define KZ_MLP_PARAMS (64 * 16 + 64 + 64 * 64 + 64 + 64 + 1)

typedef struct kz_model_s *kz_model; /* opaque; owns device memory */

/* Create a model on the current device from host weights (fp32[KZ_MLP_PARAMS];
 * NULL = all zeros).  Synchronous. */
kz_status kz_model_create(const float *weights, kz_model *out);

/* Copy the fp32 master weights back to the host (synchronous). */
kz_status kz_model_get(kz_model m, float *weights);

void kz_model_free(kz_model m);

/* Inference on device data: X device fp32[B][16], logits device fp32[B].
 * bf16 weights, fp32 accumulation.  Asynchronous on `stream`. */
kz_status kz_mlp_forward(kz_model m, const float *X, int64_t B, float *logits, void *stream);

/* Mean binary cross-entropy and its gradient with respect to the fp32 master
 * weights: X device fp32[B][16], y device fp32[B] (0 or 1); grad device
 * fp32[KZ_MLP_PARAMS] (overwritten); loss device fp32[1] (overwritten).
 * Asynchronous. */
kz_status kz_mlp_grad(kz_model m, const float *X, const float *y, int64_t B, float *grad, float *loss,
                      void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the gradient in
 * device memory; refreshes the bf16 copy.  Asynchronous. */
kz_status kz_mlp_adam(kz_model m, const float *grad, float lr, void *stream);

/*
 * Training data from the plain method: runs Jacobi sweeps on g (from its
 * current state) to the fixpoint and, in every sweep, records the features of
 * up to per_sweep_cap live edges (a seeded hash subsample) with the label
 * "this edge fails the edge rule in this sweep".  X host fp32[cap][16],
 * y host uint8[cap]; *count receives the records written.  Synchronous.
 */
kz_status kz_collect_trace(kz_graph g, int64_t per_sweep_cap, uint64_t seed, float *X, uint8_t *y,
                           int64_t cap, int64_t *count);

/* Attach a model to a graph for kz_options.schedule = KZ_SCHED_LEARNED:
 * an edge is tested in a learned round when sigmoid(score) > threshold
 * (threshold <= 0 tests every edge of the frontier).  The model must outlive
 * the graph's learned kernelizations. */
kz_status kz_attach_model(kz_graph g, kz_model m, float threshold);

#ifdef __cplusplus
}
#endif

#endif /* KZ_LEARNED_H */
