/* Learned residual potential (MLP surrogate) and its training: C ABI of libscivr.
 *
 * The paper has no network.  Its Sec. IV finds that the potential subroutine
 * (value, gradient and Hessian at every force stage) takes about 70% of the
 * run time and that the analytic form of the surface sets the speed; this part
 * of the library lets a potential carry a learned term
 *
 *   V(q) = V_analytic(q) + V_mlp(q),
 *   x = s_in * q (elementwise),  z1 = W1 x + b1,  a_l = silu(z_l),
 *   z_{l+1} = W_{l+1} a_l + b_{l+1} (l = 1, 2),  V_mlp = s_out (w4 . a3 + b4),
 *
 * (silu(z) = z / (1 + e^-z), hidden width H = 256) whose value, gradient and
 * Hessian come from BF16-input / FP32-accumulate tensor-core GEMMs batched
 * over trajectories, and which is trained on the GPU by the library's own
 * forward and backward kernels.  The analytic surface stays available as the
 * reference the network is measured against (scivr_pes_eval).
 *
 * Parameter vector theta (FP32, device): the concatenation
 *   [W1 (H x F, row-major, output index first), b1 (H), W2 (H x H), b2 (H),
 *    W3 (H x H), b3 (H), w4 (H), b4 (1)]
 * of length scivr_mlp_param_count(F, H).
 *
 * Conventions are those of scivr.h: every call is asynchronous on `stream`
 * (a cudaStream_t, NULL = legacy default stream), arguments are validated on
 * the host before any launch (SCIVR_EINVAL / SCIVR_EUNSUPPORTED with the
 * message in scivr_last_error()), and device-side failures are reported by
 * scivr_check_status().
 */
#ifndef SCIVR_MLP_H
#define SCIVR_MLP_H

#include <stdint.h>

#include "scivr.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SCIVR_MLP_HIDDEN 256   /* the only hidden width built */

/* Host description of a learned residual (all arrays FP64, host memory, read
 * during the call; the library keeps FP32 copies and BF16 tiles). */
typedef struct {
    int32_t H;              /* hidden width, SCIVR_MLP_HIDDEN */
    const double *s_in;     /* [F] input scale, x = s_in * q (> 0) */
    double s_out;           /* output scale (> 0) */
    const double *W1;       /* [H][F] */
    const double *b1;       /* [H] */
    const double *W2;       /* [H][H] */
    const double *b2;       /* [H] */
    const double *W3;       /* [H][H] */
    const double *b3;       /* [H] */
    const double *w4;       /* [H] */
    double b4;
} scivr_mlp_desc;

/* Terms selected by scivr_pes_eval. */
enum {
    SCIVR_TERMS_ALL = 0,       /* diagonal + coupling polynomial (+ learned residual is never included) */
    SCIVR_TERMS_DIAG = 1,      /* the separable diagonal (harmonic or Morse) alone */
    SCIVR_TERMS_COUPLING = 2   /* the cubic + quartic coupling polynomial alone */
};

/* Length of theta for F modes and hidden width H: H F + 2 H^2 + 4 H + 1. */
int64_t scivr_mlp_param_count(int32_t F, int32_t H);

/* Attach a learned residual to a potential, replacing any earlier one (NULL
 * detaches it).  Afterwards scivr_propagate integrates V_analytic + V_mlp
 * (split-step schedule: one batched network evaluation per force stage;
 * precision must be SCIVR_MIXED, kernel SCIVR_KERNEL_AUTO) and the other
 * scivr_mlp_* calls use these weights.  Synchronises the device.
 * Errors: SCIVR_EINVAL (NULL pes, H != 256, non-finite values, s_in or
 * s_out <= 0), SCIVR_ENOMEM, SCIVR_ECUDA. */
int scivr_pes_set_mlp(scivr_pes pes, const scivr_mlp_desc *m);

/* V_mlp, its gradient and Hessian (with respect to q) for n points.
 * q: device [n][F] FP32.  V: device [n]; g: device [n][F]; H: device
 * [n][F][F] (symmetric), or NULL for value and gradient only -- all FP32.
 * Layer 1 runs on the CUDA cores; the 256 x 256 layers run as tcgen05 GEMMs
 * with BF16 operands and FP32 accumulation.  With H, one persistent kernel
 * carries the F input-Jacobian directions as extra rows next to each point
 * (forward mode), runs the reverse pass on the point rows, and forms the
 * Hessian sum_l J_l^T diag(abar_l silu''(z_l)) J_l, all on chip.  Without H the
 * unfused kernels stage their operands in scratch allocated with
 * cudaMallocAsync on `stream` (about 3.5 n kB).  Errors: SCIVR_EINVAL (no
 * residual attached, n < 1, NULL q/V/g), SCIVR_EUNSUPPORTED (F > 9),
 * SCIVR_ENOMEM, SCIVR_ECUDA. */
int scivr_mlp_eval(scivr_pes pes, int64_t n, const float *q, float *V, float *g, float *H, void *stream);

/* Copy the current parameter vector out to / in from device memory
 * (theta: device FP32 [scivr_mlp_param_count(F, 256)]).  Setting refreshes
 * the BF16 tiles.  Errors: SCIVR_EINVAL (no residual attached, NULL). */
int scivr_mlp_get_params(scivr_pes pes, float *theta, void *stream);
int scivr_mlp_set_params(scivr_pes pes, const float *theta, void *stream);

/* Training objective of the residual alone (energy and gradient matching):
 *   L = (1/n) sum_j [ alpha (V_mlp(q_j) - Vref_j)^2 + beta |grad V_mlp(q_j) - gref_j|^2 ]
 * and its gradient with respect to theta, by one evaluation (V, grad V) and
 * one reverse pass over a forward pass that carries the single direction
 * s_in * dL/d(grad V) per point (reverse over forward mode); the weight
 * gradients of the 256 x 256 layers are split-K tcgen05 GEMMs over the
 * 2 n point rows.  q: device [n][F]; Vref: [n]; gref: [n][F]; grad: device
 * [param_count] (overwritten); loss: device [1] (overwritten) -- all FP32.
 * Allocates scratch with cudaMallocAsync on `stream`.
 * Errors: SCIVR_EINVAL (no residual, n < 1, NULL, alpha or beta < 0),
 * SCIVR_EUNSUPPORTED (F > 9), SCIVR_ENOMEM, SCIVR_ECUDA. */
int scivr_mlp_loss_grad(scivr_pes pes, int64_t n, const float *q, const float *Vref, const float *gref,
                        double alpha, double beta, float *grad, float *loss, void *stream);

/* One AdamW step on the attached residual's parameters (Loshchilov & Hutter,
 * decoupled weight decay): with bias corrections c1 = 1 - beta1^t,
 * c2 = 1 - beta2^t,
 *   m1 <- beta1 m1 + (1 - beta1) grad,  m2 <- beta2 m2 + (1 - beta2) grad^2,
 *   theta <- theta - lr (m1 / c1 / (sqrt(m2 / c2) + eps) + weight_decay theta),
 * then the BF16 tiles are refreshed.  m1, m2: device FP32 [param_count]
 * (caller-owned, zero before t = 1).  Errors: SCIVR_EINVAL (no residual, NULL,
 * t < 1, lr < 0, beta outside [0, 1)). */
int scivr_mlp_adamw(scivr_pes pes, const float *grad, float *m1, float *m2, int32_t t, double lr, double beta1,
                    double beta2, double eps, double weight_decay, void *stream);

/* Analytic potential (FP64, no learned term): V, gradient and Hessian of the
 * selected terms at n points -- the force-stage evaluation of the
 * propagation (Sec. III.A), exposed to make training targets and to measure a
 * learned residual's error.  q: device [n][F]; V: [n]; g: [n][F] (or NULL);
 * H: [n][F][F] (or NULL) -- all FP64 device.  Errors: SCIVR_EINVAL. */
int scivr_pes_eval(scivr_pes pes, int64_t n, const double *q, int32_t terms, double *V, double *g, double *H,
                   void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SCIVR_MLP_H */
