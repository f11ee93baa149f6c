// Internal declarations shared by the libscivr translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "scivr.h"
#include "scivr_mlp.h"

namespace scivr {

// Learned residual (MLP surrogate) weights on the device: FP32 masters and
// BF16 tiles of the 256 x 256 layers for the tensor-core GEMMs.
// theta is the flat parameter vector [W1 (H x F), b1, W2 (H x H), b2, W3, b3,
// w4, b4]; the named pointers point into it.
struct MlpWeightsDev {
    int H;                                   // 256 (0: no residual)
    int64_t n_params;
    float *theta;
    const float *W1, *b1, *W2, *b2, *W3, *b3, *w4, *b4;
    float s_out;
    const float *s_in;                       // [F]
    uint8_t *W2t, *W3t, *W2Tt, *W3Tt;        // BF16 tiles (refreshed whenever theta changes)
};

// Device-resident potential.  The coupling polynomial is stored in the
// Hessian-generating form used by the kernels:
//   H3[a][b] = sum_k T3[k][e(a,b)] q_k,          (cubic part of the Hessian)
//   H4[a][b] = sum_{k<=l} T4[e(k,l)][e(a,b)] q_k q_l   (quartic part)
// with e(a,b) the packed index of the upper triangle (a <= b).  By Euler's
// theorem for homogeneous polynomials, grad V3 = H3 q / 2, V3 = q.H3 q / 6,
// grad V4 = H4 q / 3 and V4 = q.H4 q / 12, so one pass over the packed
// Hessian entries yields V, grad V and H.
struct CartQ;   // cartesian.cuh

struct PesDev {
    int F, P, diag_kind;
    int kind;                        // SCIVR_PES_POLY or SCIVR_PES_CART3
    const CartQ *cart;               // SCIVR_PES_CART3: bond-vector map and force constants
    int has3, has4;
    const double *omega, *D, *a;     // [F]
    const double *T3;                // [F][P]
    const double *T4;                // [P][P]
    const float *T3f, *T4f;          // FP32 copies for the mixed-precision path
    int P4;                          // P rounded up to a multiple of 4
    const float *T3p, *T4p;          // FP32 copies [F][P4], [P][P4] with rows padded to whole
                                     // 16-byte vectors (read from global memory above F = 16)
    const float *omega_f, *D_f, *a_f;   // FP32 copies of the diagonal parameters
    MlpWeightsDev mlp;                  // mlp.H == 0: analytic surface only
};

// Kernel-side propagation parameters, passed by value.
struct PropArgs {
    int F, n_steps, n_chi, precision, kernel;
    int amplitude;                   // SCIVR_AMP_TA or SCIVR_AMP_HK
    double dt, stab_tol, ref_step;   // ref_step = sum_i gamma_i dt
    double cdrift[4], dkick[3];      // triple-jump fractions of dt
    double tdrift[4], tkick[3];      // the sub-step lengths themselves (fraction x dt)
    float tdrift_f[4], tkick_f[3];   // FP32 copies (conversions run on the FP64 pipe on GB300)
    float tdrift_lo[4], tkick_lo[3]; // their remainders (tdrift - tdrift_f ...): double-FP32 sub-steps
    float stab_tol_f;
    double gamma[SCIVR_MAX_F];
    double rg[SCIVR_MAX_F];          // sqrt(gamma)
    double irg[SCIVR_MAX_F];         // 1 / sqrt(gamma)
    double qw[SCIVR_MAX_F];          // gamma / 4
    double pw[SCIVR_MAX_F];          // 1 / (4 gamma)
    double p_eq[SCIVR_MAX_CHI * SCIVR_MAX_F];
    double q_eq[SCIVR_MAX_CHI * SCIVR_MAX_F];
};

struct FinalDev {
    double *p, *q, *S, *theta, *detM, *detA, *M, *stab;
};

struct PropLaunch {
    PesDev pes;
    PropArgs args;
    int64_t n_traj;
    const double *p0, *q0;
    double2 *amp;                 // complex double rows, or complex float rows when amp_f32
    int64_t amp_ld, chi_stride;
    int amp_f32;
    uint8_t *good;
    FinalDev fin;
};

// Amplitude sample i of a launch, stored at its precision.
__device__ __forceinline__ void amp_store(const PropLaunch &L, int64_t i, double re, double im)
{
    if (L.amp_f32) reinterpret_cast<float2 *>(L.amp)[i] = make_float2((float)re, (float)im);
    else L.amp[i] = make_double2(re, im);
}

// Amplitude rows as the Fourier steps read them: complex double, or complex float
// (the mixed path's storage).  amp[i] widens to FP64; re_f, im_f narrow one part to FP32.
struct AmpRef {
    const void *p;
    int f32;
    __host__ __device__ AmpRef offset(int64_t i) const
    {
        return AmpRef{f32 ? (const void *)(static_cast<const float2 *>(p) + i)
                          : (const void *)(static_cast<const double2 *>(p) + i), f32};
    }
#ifdef __CUDACC__
    __device__ __forceinline__ double2 operator[](int64_t i) const
    {
        if (f32) {
            const float2 v = static_cast<const float2 *>(p)[i];
            return make_double2((double)v.x, (double)v.y);
        }
        return static_cast<const double2 *>(p)[i];
    }
    __device__ __forceinline__ float re_f(int64_t i) const
    {
        return f32 ? static_cast<const float2 *>(p)[i].x : (float)static_cast<const double2 *>(p)[i].x;
    }
    __device__ __forceinline__ float im_f(int64_t i) const
    {
        return f32 ? static_cast<const float2 *>(p)[i].y : (float)static_cast<const double2 *>(p)[i].y;
    }
#endif
};

// Launchers (return cudaError_t of the launch).
cudaError_t launch_propagate(const PropLaunch &L, cudaStream_t s, int *n_launch);
cudaError_t launch_sample(int F, const double *gamma, const double *p_eq, const double *q_eq,
                          int64_t n_traj, uint64_t seed, double *p0, double *q0, double *w,
                          cudaStream_t s, int *n_launch);
cudaError_t launch_spectrum_fp64(AmpRef amp, int64_t amp_ld, const double *w,
                                 const uint8_t *good, int64_t n_traj, int n_steps, double dt,
                                 double E_min, double E_max, int n_E, double *I_out,
                                 int64_t *n_good_out, void *scratch, cudaStream_t s,
                                 int *n_launch);
size_t spectrum_fp64_scratch_bytes(int64_t n_traj, int n_steps, int n_E);
cudaError_t launch_spectrum_noalloc(AmpRef amp, int64_t amp_ld, const double *w,
                                    const uint8_t *good, int64_t n_traj, int n_steps, double dt,
                                    double E_min, double E_max, int n_E, double *I_out,
                                    int64_t *n_good_out, cudaStream_t s, int *n_launch);
int spectrum_noalloc_max_energies();
size_t spectrum_hk_scratch_bytes(int64_t n_traj, int n_steps);
cudaError_t launch_spectrum_hk(const double2 *amp, int64_t amp_ld, const uint8_t *good, int64_t n_traj, int n_steps,
                               double dt, double E_min, double E_max, int n_E, double *I_out, double2 *C_out,
                               int64_t *n_good_out, void *scratch, cudaStream_t s, int *n_launch);
int spectrum_czt_max_samples();
constexpr int kCztMaxEnergies = 12288;   // per-CTA weighted sums beside the 128 KB transform buffer
size_t spectrum_czt_scratch_bytes(int64_t n_traj, int n_steps, int n_E);
cudaError_t launch_spectrum_czt(AmpRef amp, int64_t amp_ld, const double *w, const uint8_t *good,
                                int64_t n_traj, int n_steps, double dt, double E_min, double E_max, int n_E,
                                double *I_out, int64_t *n_good_out, void *scratch, cudaStream_t s, int *n_launch);
int ft_tc_digits(int ft_mode);
size_t spectrum_tc_scratch_bytes(int ft_mode, int64_t n_traj, int n_steps, int n_E);
cudaError_t launch_spectrum_tc(int ft_mode, AmpRef amp, int64_t amp_ld, const double *w,
                               const uint8_t *good, int64_t n_traj, int n_steps, double dt, double E_min,
                               double E_max, int n_E, double *I_out, int64_t *n_good_out, void *scratch,
                               cudaStream_t s, int *n_launch);
cudaError_t launch_wait_selftest(double seconds, cudaStream_t s);
cudaError_t read_and_clear_status(int *status);
cudaError_t read_and_clear_status_mlp(int *status);
size_t mlp_eval_scratch_bytes(int F, int64_t n, bool hess);
size_t mlp_train_scratch_bytes(int F, int64_t n);
cudaError_t mlp_prepare();   // kernel attributes (current device); call before the first launch
cudaError_t mlp_eval(const MlpWeightsDev &w, int F, int64_t n, const float *q, float *V, float *g, float *H,
                     void *scratch, cudaStream_t s, int *n_launch);   // H == NULL: V and g only
cudaError_t mlp_loss_grad(const MlpWeightsDev &w, int F, int64_t n, const float *q, const float *Vref,
                          const float *gref, float alpha, float beta, float *grad, float *loss, void *scratch,
                          cudaStream_t s, int *n_launch);
cudaError_t mlp_tile_weights(const MlpWeightsDev &w, cudaStream_t s);   // 4 launches
cudaError_t mlp_adamw(const MlpWeightsDev &w, const float *grad, float *m1, float *m2, float lr, float beta1,
                      float beta2, float eps, float wd, float c1, float c2, cudaStream_t s);   // 5 launches
// Split-step propagation on a potential with a learned residual (pes.mlp.H != 0).
cudaError_t launch_propagate_mlp(const PropLaunch &L, cudaStream_t s, int *n_launch);
cudaError_t launch_pes_eval(const PesDev &pes, int64_t n, const double *q, int terms, double *V, double *g,
                            double *H, cudaStream_t s);

bool propagate_supported(int F, int precision, int kernel);
int prepare_propagate(scivr_pes pes, const scivr_prop_params *prm, int64_t n_traj, const double *p0,
                      const double *q0, void *amp, int64_t amp_ld, uint8_t *good,
                      const scivr_final_state *fin, PropLaunch *out);
int check_spectrum_args(const void *amp, int64_t amp_ld, int32_t amp_prec, const double *w, const uint8_t *good,
                        int64_t n_traj, int32_t n_steps, double dt, double E_min, double E_max, int32_t n_E,
                        int32_t ft_mode, const double *I_out,
                        const char *who);
int set_error(int code, const char *msg);
void clear_error();
void count_launches(int n);
int cuda_error(cudaError_t e, const char *where);
// Batched persistent lane-group launch for mixed precision; warps must be one of
// batch_warp_candidates(F).
cudaError_t launch_group_batch_mixed(int F, int warps, const PropLaunch *items, const int2 *work, int n_work,
                                     int *counter, int n_sm, cudaStream_t s);
int batch_warp_candidates(int F, int *out);   // returns the count (<= 2)
// One persistent launch for molecules of several F (the batch recipe's classes).
bool multi_launch_holds(int F);
int multi_launch_tile(int F);                  // trajectories per work item
cudaError_t launch_group_batch_multi(const PropLaunch *items, const int2 *work, int n_work, int *counter, int n_sm,
                                     cudaStream_t s);

// Lanes per trajectory of the mixed-precision lane-group kernels: every mode and at
// most two monodromy columns per lane -- 8 lanes up to F = 4, 16 up to F = 9 (at F = 9
// two lanes hold a second column, so a warp carries two trajectories), 32 above.
__host__ __device__ constexpr int mixed_group_lanes(int F) { return 2 * F <= 8 ? 8 : (F <= 9 ? 16 : 32); }

// log <chi_x|p0_j, q0_j> (Eq. coherent_state with unit-norm states).
template <int F>
__device__ __forceinline__ void chi_log_overlap_at(const PropArgs &A, const double *p0, const double *q0,
                                                   int64_t n, int64_t j, int x, double &re, double &im)
{
    re = 0.0;
    im = 0.0;
#pragma unroll
    for (int a = 0; a < F; ++a) {
        const double pa = p0[a * n + j], qa = q0[a * n + j];
        const double dq = A.q_eq[x * F + a] - qa, dp = A.p_eq[x * F + a] - pa;
        re = fma(-A.qw[a] * dq, dq, re);
        re = fma(-A.pw[a] * dp, dp, re);
        im = fma(0.5 * (A.p_eq[x * F + a] + pa), dq, im);
    }
}

// The logarithm re0 + i im0 that the Herman-Kluk summand of reference state x
// divides by.  The summand is C e^{iS} <chi_x|p_t q_t> <p0 q0|chi_x> / |<p0 q0|chi_0>|^2:
// the initial conditions are drawn from the Husimi density of the first reference
// state, so that density's inverse is every state's importance weight.  Hence
// im0 = Im log <chi_x|p0 q0> and re0 = 2 Re log <chi_0|p0 q0> - Re log <chi_x|p0 q0>
// (for x = 0 exactly Re log <chi_0|p0 q0>).  Call it for x = 0, 1, ... in order:
// the x = 0 call stores Re log <chi_0|p0 q0> in re00 for the later ones.
template <int F>
__device__ __forceinline__ void chi_log_overlap0(const PropArgs &A, const double *p0, const double *q0,
                                                 int64_t n, int64_t j, int x, double &re00, double &re0,
                                                 double &im0)
{
    chi_log_overlap_at<F>(A, p0, q0, n, j, x, re0, im0);
    if (x == 0) re00 = re0;
    else re0 = 2.0 * re00 - re0;
}

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kInvTwoPi = 0.15915494309189533576888376337251;

}  // namespace scivr

struct scivr_pes_s {
    scivr::PesDev dev;
    void *blob;          // single device allocation holding all arrays
    void *mlp_blob;      // learned-residual weights and tiles (or NULL)
};
