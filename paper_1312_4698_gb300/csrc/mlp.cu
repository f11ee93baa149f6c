// Learned-residual potential (MLP surrogate): batched V, grad V and Hessian,
// and the gradient of its training objective, with BF16-in / FP32-accumulate
// tcgen05 GEMMs.
//
// Network (hidden width 256, F <= 9 inputs):
//   x = s_in q,  z1 = W1 x + b1,  a_l = silu(z_l),  z_{l+1} = W_{l+1} a_l + b_{l+1},
//   V_mlp = s_out (w4 . a3 + b4).
//
// Evaluation.  The input Jacobians J_l = dz_l/dx travel forward as F extra
// "tangent" rows per point (row k of layer l+1's input is silu'(z_l) J_l[:, k]),
// so one GEMM per layer serves the value and all F directions.  The reverse
// pass (point rows only) gives abar_l = dy/da_l; then
//   grad V = s_out s_in * W1^T (abar_1 silu'(z1)),
//   Hess V = s_out diag(s_in) [sum_l J_l^T diag(abar_l silu''(z_l)) J_l] diag(s_in).
// With the Hessian, k_mlp_fused keeps a tile of 12 points x (1 + F) rows on
// chip from input to outputs.  Without it (the training pass and value +
// gradient requests) a point has a single row and the unfused kernels below
// stage their operands in HBM.
//
// Training objective L = (1/n) sum_j alpha (V_j - Vref_j)^2 + beta |g_j - gref_j|^2.
// With e_j = 2 alpha (V_j - Vref_j) / n and u_j = 2 beta (g_j - gref_j) / n held
// fixed, dL/dtheta = s_out sum_j d/dtheta [e_j y_j + D_{xd_j} y_j] with the
// direction xd_j = s_in * u_j (reverse mode over a forward-mode pass): point
// row 2j carries a_l, row 2j+1 carries the tangent adot_l = silu'(z_l) zdot_l.
// Reverse:  zbar = abar silu'(z) + adotbar silu''(z) zdot,  zdotbar = adotbar silu'(z),
//           Wbar_l = sum_rows [zbar; zdotbar] [a_{l-1}; adot_{l-1}]^T,
//           [abar; adotbar]_{l-1} = W_l^T [zbar; zdotbar],  bbar_l = sum_j zbar.
// The weight gradients of the 256 x 256 layers are split-K GEMMs over the
// 2 n rows, so the activation kernels also write their output transposed
// (hidden index as the tile row, the point row as k).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "tc_common.cuh"

namespace scivr {
namespace mlp {

using namespace tc;
constexpr int HW = 256;                 // hidden width
constexpr int KT_H = HW / BK;           // k tiles of a 256-wide operand
constexpr int kMaxF = 9;
constexpr int TSMEM = BM * HW * 2;      // one 128 x 256 BF16 tile staged in shared memory

__device__ __forceinline__ void silu3(float z, float &f, float &f1, float &f2)
{
    const float s = 1.0f / (1.0f + __expf(-z));
    f = z * s;
    f1 = s * (1.0f + z * (1.0f - s));
    f2 = s * (1.0f - s) * (2.0f + z * (1.0f - 2.0f * s));
}

// ---------------------------------------------------------------- GEMM
// C[m][n] = sum_k A[m][k] B[n][k] over k tiles [z kt_split, (z+1) kt_split) of
// n_kt (blockIdx.z = z).  A and B are pre-tiled (canonical K-major: A blocks
// of 128 rows x 32 k, B blocks of 256 x 32, block (row block, k tile) at
// (row_block n_kt + k_tile) x block bytes); C is FP32 row-major with leading
// dimension ldc, split z at C + z c_split; rows >= m_valid are not written.
// grid = (N / 256, M / 128, splits), 128 threads.
__global__ void __launch_bounds__(128, 1)
    k_gemm(const uint8_t *__restrict__ At, const uint8_t *__restrict__ Bt, int n_kt, int kt_split,
           float *__restrict__ C, int64_t ldc, int64_t m_valid, int64_t c_split)
{
    constexpr int STAGES = 6;
    constexpr int STAGE = TILE_A + TILE_B;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nt = blockIdx.x;
    const int64_t mt = blockIdx.y;
    const int kt0 = blockIdx.z * kt_split;
    const int cnt = (n_kt - kt0) < kt_split ? (n_kt - kt0) : kt_split;   // >= 1 by the grid
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"(256) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint8_t *Ablk = At + ((size_t)mt * n_kt + kt0) * TILE_A;
    const uint8_t *Bblk = Bt + ((size_t)nt * n_kt + kt0) * TILE_B;
    if (warp == 0 && lane == 0) {
        int issued = 0;
        for (int kt = 0; kt < cnt; ++kt) {
            const int s = kt % STAGES, use = kt / STAGES;
            if (use > 0 && !mbar_wait(&empty_bar[s], (use - 1) & 1, kWaitLimitCycles)) { atomicExch(&abort_flag, 1); break; }
            if (*(volatile int *)&abort_flag) break;
            uint8_t *sa = smem + s * STAGE;
            mbar_expect_tx(&full_bar[s], STAGE);
            bulk_g2s(sa, Ablk + (size_t)kt * TILE_A, TILE_A, &full_bar[s]);
            bulk_g2s(sa + TILE_A, Bblk + (size_t)kt * TILE_B, TILE_B, &full_bar[s]);
            issued = kt + 1;
        }
        // do not leave the CTA with copies still landing in its shared memory
        for (int kt = issued - STAGES > 0 ? issued - STAGES : 0; kt < issued; ++kt)
            mbar_wait(&full_bar[kt % STAGES], (kt / STAGES) & 1, kWaitLimitCycles);
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = idesc_bf16(BM, BN);
        for (int kt = 0; kt < cnt; ++kt) {
            const int s = kt % STAGES;
            if (!mbar_wait(&full_bar[s], (kt / STAGES) & 1, kWaitLimitCycles) || *(volatile int *)&abort_flag) {
                atomicExch(&abort_flag, 1);
                break;
            }
            tc_fence_after();
            const uint32_t sa = su32(smem + s * STAGE), sb = sa + TILE_A;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks)
                umma(tmem, sdesc(sa + ks * 2 * LBO), sdesc(sb + ks * 2 * LBO), idesc, (kt | ks) != 0);
            umma_commit(&empty_bar[s]);
        }
        umma_commit(&done_bar);
    }
    __syncwarp();
    const bool ok = mbar_wait(&done_bar, 0, kWaitLimitCycles) && !*(volatile int *)&abort_flag;
    tc_fence_after();
    __syncwarp();
    const int row = warp * 32 + lane;
    const int64_t grow = mt * BM + row;
    float *Cz = C + (int64_t)blockIdx.z * c_split;
#pragma unroll 1
    for (int ch = 0; ch < BN / 32; ++ch) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + ch * 32, v);
        tmem_wait_ld();
        if (ok && grow < m_valid) {
            float4 *dst = reinterpret_cast<float4 *>(Cz + grow * ldc + (int64_t)nt * BN + ch * 32);
#pragma unroll
            for (int i = 0; i < 8; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
    }
}

constexpr int GEMM_SMEM = 6 * (TILE_A + TILE_B) + 1024;

// ---------------------------------------------------------------- tiling helpers
// Byte address of element (r, k) of a tiled operand with RB-row blocks and n_kt k tiles.
template <int RB>
__device__ __forceinline__ uint8_t *tile_addr(uint8_t *base, int n_kt, int64_t r, int64_t k)
{
    constexpr int BLK = RB * BK * 2;
    return base + (((r / RB) * n_kt + k / BK) * (int64_t)BLK) + canon_off((int)(r % RB), (int)(k % BK));
}

// Write 8 consecutive k-values (k0 a multiple of 8) of row r.
template <int RB>
__device__ __forceinline__ void put8(uint8_t *base, int n_kt, int64_t r, int64_t k0, const float (&v)[8])
{
    __nv_bfloat16 h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) h[i] = __float2bfloat16_rn(v[i]);
    *reinterpret_cast<uint4 *>(tile_addr<RB>(base, n_kt, r, k0)) = *reinterpret_cast<const uint4 *>(h);
}

// A 128 x 256 BF16 tile T (row-major, shared memory) of 128-row block `tile`:
// rows -> A operand with K = 256 (row = point row, k = hidden index).
__device__ __forceinline__ void store_rows(const __nv_bfloat16 *T, uint8_t *X, int64_t tile)
{
    for (int idx = threadIdx.x; idx < BM * (HW / 8); idx += blockDim.x) {
        const int rr = idx % BM, ch = idx / BM;
        *reinterpret_cast<uint4 *>(tile_addr<BM>(X, KT_H, tile * BM + rr, ch * 8)) =
            *reinterpret_cast<const uint4 *>(T + rr * HW + ch * 8);
    }
}

// Same tile transposed: row = hidden index (RB-row blocks), k = point row (n_kt k tiles in all).
template <int RB>
__device__ __forceinline__ void store_cols(const __nv_bfloat16 *T, uint8_t *XT, int n_kt, int64_t tile)
{
    for (int idx = threadIdx.x; idx < HW * (BM / 8); idx += blockDim.x) {
        const int i = idx % HW, r0 = (idx / HW) * 8;
        __nv_bfloat16 h[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) h[k] = T[(r0 + k) * HW + i];
        *reinterpret_cast<uint4 *>(tile_addr<RB>(XT, n_kt, i, tile * BM + r0)) = *reinterpret_cast<const uint4 *>(h);
    }
}

// Weight matrix W [256 out][256 in] (FP32 row-major) -> B tiles of W (forward:
// rows = out, k = in) or of W^T (reverse: rows = in, k = out).
__global__ void k_tile_weight(const float *__restrict__ W, int transpose, uint8_t *__restrict__ Bt)
{
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;   // (row, chunk) over 256 x 32
    if (gid >= HW * (HW / 8)) return;
    const int r = gid / (HW / 8), k0 = (gid % (HW / 8)) * 8;
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = transpose ? W[(k0 + i) * HW + r] : W[r * HW + k0 + i];
    put8<256>(Bt, KT_H, r, k0, v);
}

struct MlpDev {
    int F, spt, rows_per_sample;    // points per 128-row tile, rows per point
    const float *W1, *b1, *W2, *b2, *W3, *b3, *w4, *b4;   // FP32 master copies (device)
    float s_out;
    const float *s_in;              // [F]
    const uint8_t *W2t, *W3t, *W2Tt, *W3Tt;               // BF16 B tiles
};

__device__ __forceinline__ int64_t point_row(const MlpDev &m, int64_t b)
{
    return (b / m.spt) * BM + (b % m.spt) * m.rows_per_sample;
}

// ---------------------------------------------------------------- evaluation
// Layer 1 (K = F, CUDA cores) for one 128-row tile: writes the layer-2 input
// rows (a1, and the tangents silu'(z1) W1[:, k] when rows_per_sample = F + 1)
// as A tiles, and keeps z1 for the reverse pass.  Dynamic shared memory:
// spt x 256 floats.
__global__ void k_layer1(MlpDev m, int64_t n, const float *__restrict__ q, uint8_t *__restrict__ X2,
                         float *__restrict__ Z1)
{
    extern __shared__ float zs[];   // [spt][HW]
    const int64_t tile = blockIdx.x;
    const int F = m.F, R = m.rows_per_sample, spt = m.spt;
    for (int idx = threadIdx.x; idx < spt * HW; idx += blockDim.x) {
        const int s = idx / HW, o = idx % HW;
        const int64_t b = tile * spt + s;
        float z = m.b1[o];
        if (b < n)
            for (int i = 0; i < F; ++i) z = fmaf(m.W1[o * F + i], m.s_in[i] * q[b * F + i], z);
        zs[s * HW + o] = z;
        if (b < n) Z1[b * HW + o] = z;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < BM * (HW / 8); idx += blockDim.x) {
        const int rr = idx % BM, ch = idx / BM;
        const int s = rr / R, k = rr % R;
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int o = ch * 8 + i;
            float val = 0.0f;
            if (s < spt && tile * spt + s < n) {
                float f, f1, f2;
                silu3(zs[s * HW + o], f, f1, f2);
                val = k == 0 ? f : f1 * m.W1[o * F + (k - 1)];
            }
            v[i] = val;
        }
        put8<BM>(X2, KT_H, tile * BM + rr, ch * 8, v);
    }
}

// Activation of a hidden layer for one tile: C holds z - b (point rows) and the
// tangents' dz (tangent rows); writes the next layer's input rows.  With XT
// set, the tile is also written transposed as a B operand (training).
// Dynamic shared memory: TSMEM.
__global__ void k_hidden_act(MlpDev m, int64_t n, const float *__restrict__ Cz, const float *__restrict__ bias,
                             uint8_t *__restrict__ Xn, uint8_t *__restrict__ XT, int n_kt_rows)
{
    extern __shared__ __align__(16) __nv_bfloat16 T[];   // [BM][HW]
    const int64_t tile = blockIdx.x;
    const int R = m.rows_per_sample, spt = m.spt;
    for (int idx = threadIdx.x; idx < BM * HW; idx += blockDim.x) {
        const int rr = idx / HW, o = idx % HW;
        const int s = rr / R, k = rr % R;
        float val = 0.0f;
        if (s < spt && tile * spt + s < n) {
            const int64_t prow = tile * BM + s * R;
            float f, f1, f2;
            silu3(Cz[prow * HW + o] + bias[o], f, f1, f2);
            val = k == 0 ? f : f1 * Cz[(tile * BM + rr) * HW + o];
        }
        T[idx] = __float2bfloat16_rn(val);
    }
    __syncthreads();
    store_rows(T, Xn, tile);
    if (XT) store_cols<256>(T, XT, n_kt_rows, tile);
}

// Output layer and the first reverse step: V = s_out (w4 . a3 + b4) and
// delta3 = w4 silu'(z3) as A rows (one row per point) of the reverse GEMM.
__global__ void k_output(MlpDev m, int64_t n, const float *__restrict__ C3, float *__restrict__ V,
                         uint8_t *__restrict__ D3)
{
    const int64_t b = blockIdx.x;            // one CTA (256 threads) per point
    const int o = threadIdx.x;
    float f = 0.0f, f1 = 0.0f, f2;
    if (b < n) silu3(C3[point_row(m, b) * HW + o] + m.b3[o], f, f1, f2);
    float part = m.w4[o] * f;
    __shared__ float red[8];
    __shared__ float dv[HW];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((o & 31) == 0) red[o >> 5] = part;
    dv[o] = m.w4[o] * f1;
    __syncthreads();
    if (o == 0 && b < n) {
        float y = *m.b4;
        for (int w = 0; w < 8; ++w) y += red[w];
        V[b] = m.s_out * y;
    }
    if (o < HW / 8) {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = b < n ? dv[o * 8 + i] : 0.0f;
        put8<BM>(D3, KT_H, b, o * 8, v);
    }
}

// Reverse activation: delta = abar silu'(z) for the point rows (z from C + bias).
__global__ void k_backward_act(MlpDev m, int64_t n, const float *__restrict__ Abar, const float *__restrict__ Cz,
                               const float *__restrict__ bias, uint8_t *__restrict__ Dn)
{
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n_pad = (n + BM - 1) / BM * BM;
    if (gid >= n_pad * (HW / 8)) return;
    const int64_t b = gid / (HW / 8);
    const int ch = (int)(gid % (HW / 8));
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int o = ch * 8 + i;
        float val = 0.0f;
        if (b < n) {
            float f, f1, f2;
            silu3(Cz[point_row(m, b) * HW + o] + bias[o], f, f1, f2);
            val = Abar[b * HW + o] * f1;
        }
        v[i] = val;
    }
    put8<BM>(Dn, KT_H, b, ch * 8, v);
}

// Gradient of one point per warp (value-only rows: grad V = s_out s_in W1^T (abar1 silu'(z1))).
template <int F>
__global__ void k_grad(MlpDev m, int64_t n, const float *__restrict__ Z1, const float *__restrict__ Abar1,
                       float *__restrict__ g)
{
    const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= n) return;
    float gacc[F];
#pragma unroll
    for (int k = 0; k < F; ++k) gacc[k] = 0.0f;
    for (int j = 0; j < HW / 32; ++j) {
        const int i = lane + 32 * j;
        float f, f1, f2;
        silu3(Z1[b * HW + i], f, f1, f2);
        const float d1 = Abar1[b * HW + i] * f1;
#pragma unroll
        for (int k = 0; k < F; ++k) gacc[k] = fmaf(m.W1[i * F + k], d1, gacc[k]);
    }
#pragma unroll
    for (int k = 0; k < F; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) gacc[k] += __shfl_xor_sync(0xffffffffu, gacc[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < F; ++k) g[b * F + k] = m.s_out * m.s_in[k] * gacc[k];
}

// ---------------------------------------------------------------- training
// Row layout: point j of tile t = j / 64 owns rows 2 (j mod 64) (values) and
// 2 (j mod 64) + 1 (tangent) of the tile.  Per-tile partial sums of the
// small parameter gradients: [W1 (256 F) | b1 | b2 | b3 | w4 (256 each) | b4].
constexpr int TR_SPT = BM / 2;

__host__ __device__ constexpr int part_len(int F) { return HW * F + 4 * HW + 1; }

// Loss terms, the fixed direction xd = s_in u, and layer 1 of the value and
// tangent rows.  Dynamic shared memory: TSMEM + 2 TR_SPT kMaxF floats.
__global__ void k_tr_layer1(MlpDev m, int64_t n, const float *__restrict__ q, const float *__restrict__ V1,
                            const float *__restrict__ g1, const float *__restrict__ Vref,
                            const float *__restrict__ gref, float alpha, float beta, float inv_n,
                            uint8_t *__restrict__ X2, uint8_t *__restrict__ X2T, int n_kt_rows,
                            float *__restrict__ Z1, float *__restrict__ Zd1, float *__restrict__ X0,
                            float *__restrict__ Xd0, float *__restrict__ ebar, float *__restrict__ loss)
{
    extern __shared__ __align__(16) uint8_t sm[];
    __nv_bfloat16 *T = reinterpret_cast<__nv_bfloat16 *>(sm);
    float *xs = reinterpret_cast<float *>(sm + TSMEM);   // [TR_SPT][kMaxF]
    float *xds = xs + TR_SPT * kMaxF;
    const int64_t tile = blockIdx.x;
    const int F = m.F;
    if (threadIdx.x < TR_SPT) {
        const int s = threadIdx.x;
        const int64_t b = tile * TR_SPT + s;
        float lp = 0.0f;
        if (b < n) {
            const float dv = V1[b] - Vref[b];
            lp = alpha * dv * dv;
            ebar[b] = m.s_out * 2.0f * alpha * dv * inv_n;
            for (int k = 0; k < F; ++k) {
                const float dg = g1[b * F + k] - gref[b * F + k];
                lp = fmaf(beta * dg, dg, lp);
                const float x = m.s_in[k] * q[b * F + k];
                const float xd = m.s_in[k] * 2.0f * beta * dg * inv_n;
                xs[s * kMaxF + k] = x;
                xds[s * kMaxF + k] = xd;
                X0[b * F + k] = x;
                Xd0[b * F + k] = xd;
            }
        } else {
            for (int k = 0; k < F; ++k) xs[s * kMaxF + k] = xds[s * kMaxF + k] = 0.0f;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) lp += __shfl_xor_sync(0xffffffffu, lp, off);
        if ((threadIdx.x & 31) == 0) atomicAdd(loss, lp * inv_n);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < TR_SPT * HW; idx += blockDim.x) {
        const int s = idx / HW, o = idx % HW;
        const int64_t b = tile * TR_SPT + s;
        float z = m.b1[o], zd = 0.0f;
        for (int k = 0; k < F; ++k) {
            const float w = m.W1[o * F + k];
            z = fmaf(w, xs[s * kMaxF + k], z);
            zd = fmaf(w, xds[s * kMaxF + k], zd);
        }
        float f = 0.0f, f1 = 0.0f, f2;
        if (b < n) {
            Z1[b * HW + o] = z;
            Zd1[b * HW + o] = zd;
            silu3(z, f, f1, f2);
        }
        T[(2 * s) * HW + o] = __float2bfloat16_rn(f);
        T[(2 * s + 1) * HW + o] = __float2bfloat16_rn(f1 * zd);
    }
    __syncthreads();
    store_rows(T, X2, tile);
    store_cols<256>(T, X2T, n_kt_rows, tile);
}

// Output layer reverse step: zbar3, zdotbar3 (A rows and transposed A tiles)
// and the partial sums of the w4, b3 and b4 gradients.  Thread = hidden unit.
__global__ void __launch_bounds__(256) k_tr_out(MlpDev m, int64_t n, const float *__restrict__ C3,
                                                const float *__restrict__ ebar, uint8_t *__restrict__ D3,
                                                uint8_t *__restrict__ D3T, int n_kt_rows, float *__restrict__ part)
{
    extern __shared__ __align__(16) __nv_bfloat16 T[];
    const int64_t tile = blockIdx.x;
    const int o = threadIdx.x;
    const float w4 = m.w4[o], b3 = m.b3[o], at = m.s_out * w4;
    float acc_w4 = 0.0f, acc_b3 = 0.0f, acc_b4 = 0.0f;
    for (int s = 0; s < TR_SPT; ++s) {
        const int64_t b = tile * TR_SPT + s;
        float zb = 0.0f, zdb = 0.0f;
        if (b < n) {
            const int64_t r = tile * BM + 2 * s;
            const float zd = C3[(r + 1) * HW + o];
            float f, f1, f2;
            silu3(C3[r * HW + o] + b3, f, f1, f2);
            const float eb = ebar[b];
            zb = fmaf(eb * w4, f1, at * f2 * zd);
            zdb = at * f1;
            acc_w4 = fmaf(eb, f, fmaf(m.s_out * f1, zd, acc_w4));
            acc_b3 += zb;
            acc_b4 += eb;
        }
        T[(2 * s) * HW + o] = __float2bfloat16_rn(zb);
        T[(2 * s + 1) * HW + o] = __float2bfloat16_rn(zdb);
    }
    float *P = part + tile * part_len(m.F);
    const int F = m.F;
    P[HW * F + 3 * HW + o] = acc_w4;
    P[HW * F + 2 * HW + o] = acc_b3;
    if (o == 0) P[HW * F + 4 * HW] = acc_b4;
    __syncthreads();
    store_rows(T, D3, tile);
    store_cols<BM>(T, D3T, n_kt_rows, tile);
}

// Hidden layer 2 reverse step (from the adjoints Ab = D3 W3 of layer 3's inputs).
__global__ void __launch_bounds__(256) k_tr_back(MlpDev m, int64_t n, const float *__restrict__ Ab,
                                                 const float *__restrict__ C2, uint8_t *__restrict__ D2,
                                                 uint8_t *__restrict__ D2T, int n_kt_rows, float *__restrict__ part)
{
    extern __shared__ __align__(16) __nv_bfloat16 T[];
    const int64_t tile = blockIdx.x;
    const int o = threadIdx.x;
    const float b2 = m.b2[o];
    float acc_b2 = 0.0f;
    for (int s = 0; s < TR_SPT; ++s) {
        const int64_t b = tile * TR_SPT + s;
        float zb = 0.0f, zdb = 0.0f;
        if (b < n) {
            const int64_t r = tile * BM + 2 * s;
            const float zd = C2[(r + 1) * HW + o];
            float f, f1, f2;
            silu3(C2[r * HW + o] + b2, f, f1, f2);
            const float ab = Ab[r * HW + o], adb = Ab[(r + 1) * HW + o];
            zb = fmaf(ab, f1, adb * f2 * zd);
            zdb = adb * f1;
            acc_b2 += zb;
        }
        T[(2 * s) * HW + o] = __float2bfloat16_rn(zb);
        T[(2 * s + 1) * HW + o] = __float2bfloat16_rn(zdb);
    }
    part[tile * part_len(m.F) + HW * m.F + HW + o] = acc_b2;
    __syncthreads();
    store_rows(T, D2, tile);
    store_cols<BM>(T, D2T, n_kt_rows, tile);
}

// Layer 1 reverse step: partial sums of the W1 and b1 gradients.
template <int F>
__global__ void __launch_bounds__(256) k_tr_back1(MlpDev m, int64_t n, const float *__restrict__ Ab,
                                                  const float *__restrict__ Z1, const float *__restrict__ Zd1,
                                                  const float *__restrict__ X0, const float *__restrict__ Xd0,
                                                  float *__restrict__ part)
{
    const int64_t tile = blockIdx.x;
    const int o = threadIdx.x;
    float accW[F], acc_b1 = 0.0f;
#pragma unroll
    for (int k = 0; k < F; ++k) accW[k] = 0.0f;
    for (int s = 0; s < TR_SPT; ++s) {
        const int64_t b = tile * TR_SPT + s;
        if (b >= n) break;
        const int64_t r = tile * BM + 2 * s;
        float f, f1, f2;
        const float zd = Zd1[b * HW + o];
        silu3(Z1[b * HW + o], f, f1, f2);
        const float ab = Ab[r * HW + o], adb = Ab[(r + 1) * HW + o];
        const float zb = fmaf(ab, f1, adb * f2 * zd);
        const float zdb = adb * f1;
        acc_b1 += zb;
#pragma unroll
        for (int k = 0; k < F; ++k) accW[k] = fmaf(zb, X0[b * F + k], fmaf(zdb, Xd0[b * F + k], accW[k]));
    }
    float *P = part + tile * part_len(F);
#pragma unroll
    for (int k = 0; k < F; ++k) P[o * F + k] = accW[k];
    P[HW * F + o] = acc_b1;
}

// Sum the partials into the flat gradient [W1 | b1 | W2 | b2 | W3 | b3 | w4 | b4].
__global__ void k_tr_reduce(int F, int n_tiles, const float *__restrict__ part, int n_split,
                            const float *__restrict__ GW2, const float *__restrict__ GW3, float *__restrict__ grad)
{
    const int64_t n_par = (int64_t)HW * F + 2 * HW * HW + 4 * HW + 1;
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n_par) return;
    const int64_t oW2 = (int64_t)HW * F + HW, ob2 = oW2 + HW * HW, oW3 = ob2 + HW, ob3 = oW3 + HW * HW;
    const int64_t ow4 = ob3 + HW, ob4 = ow4 + HW;
    const int PL = part_len(F);
    float acc = 0.0f;
    if ((p >= oW2 && p < ob2) || (p >= oW3 && p < ob3)) {
        const float *G = p < ob2 ? GW2 + (p - oW2) : GW3 + (p - oW3);
        for (int s = 0; s < n_split; ++s) acc += G[(int64_t)s * HW * HW];
    } else {
        int idx;
        if (p < oW2) idx = (int)p;                                    // W1, b1
        else if (p < oW3) idx = HW * F + HW + (int)(p - ob2);         // b2
        else if (p < ow4) idx = HW * F + 2 * HW + (int)(p - ob3);     // b3
        else if (p < ob4) idx = HW * F + 3 * HW + (int)(p - ow4);     // w4
        else idx = HW * F + 4 * HW;                                   // b4
        for (int t = 0; t < n_tiles; ++t) acc += part[(int64_t)t * PL + idx];
    }
    grad[p] = acc;
}

__global__ void k_adamw(float *__restrict__ theta, const float *__restrict__ grad, float *__restrict__ m1,
                        float *__restrict__ m2, int64_t n, float lr, float beta1, float beta2, float eps, float wd,
                        float c1, float c2)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gr = grad[i];
    const float a = fmaf(beta1, m1[i], (1.0f - beta1) * gr);
    const float v = fmaf(beta2, m2[i], (1.0f - beta2) * gr * gr);
    m1[i] = a;
    m2[i] = v;
    const float step = (a / c1) / (sqrtf(v / c2) + eps);
    theta[i] -= lr * (step + wd * theta[i]);
}

// ---------------------------------------------------------------- fused evaluation
// V, grad V and the Hessian with every intermediate on chip.  A persistent CTA
// (one per SM: 512 TMEM columns, ~225 KB of shared memory) walks 128-row tiles
// of 12 points x (1 + F) rows.  Per tile, six tensor-core products:
//   layer 1 (CUDA cores)            -> A tile X2
//   X2 W2^T -> TMEM[0:256)             epilogue: X3 = [silu(z2); silu'(z2) J2] -> A tile
//   X3 W3^T -> TMEM[256:512)           epilogue: V, c3 = w4 silu''(z3); Gram operands
//   (c3 J3) J3^T -> TMEM[256:368)      block-diagonal Gram product: the layer-3 Hessian
//                                      term of every point at once; epilogue: delta3 -> A tile
//   D3 W3 -> TMEM[256:512)             epilogue: c2 = abar2 silu''(z2); Gram operands (J2 is
//                                      still in TMEM[0:256) next to z2 - b2 of the value rows)
//   (c2 J2) J2^T -> TMEM[256:368)      layer-2 Hessian term; epilogue: delta2 -> A tile
//   D2 W2 -> TMEM[256:512)             epilogue: grad V and the layer-1 term W1^T diag(c1) W1
// The four weight products stream BF16 weight tiles (16 KB k-blocks, 3-stage
// ring, cp.async.bulk); the two Gram products take FP16 operands written by
// the compute warps (c J rows into the A tile, the F tangent rows of every
// point packed as the 12 F x 256 B operand).  Warp roles: warps 0-7 compute
// (tile row r = TMEM lane r is shared by warps r/32 and r/32 + 4, which take
// the column halves), warp 8 streams weights, warp 9 issues tcgen05.mma.
constexpr int FU_STAGES = 3;
constexpr int FU_NC = 256;                        // compute threads
constexpr int FU_SPT = 12;                        // points per tile (F <= 9: 12 (F+1) <= 120 rows)
constexpr int FU_PS = HW + 4;                     // padded row stride of the per-point buffers
constexpr int FU_BUF = FU_SPT * FU_PS * 4;
constexpr int FU_NG = 112;                        // Gram B rows at most: 12 x 9 tangent rows, padded
constexpr int FU_GBLK = FU_NG * BK * 2;           // one 32-k block of the Gram B operand
constexpr int FU_SCS = 68;                        // row stride (floats) of the Gram read-out scratch
constexpr int FU_O_A = 0;                         // A tile: 8 k-blocks of 128 x 32 (BF16 or FP16)
constexpr int FU_O_B = FU_O_A + BM * HW * 2;      // weight ring
constexpr int FU_O_G = FU_O_B + FU_STAGES * TILE_B;   // Gram B operand, then the read-out scratch
constexpr int FU_O_P = FU_O_G + KT_H * FU_GBLK;
constexpr int FU_O_Q = FU_O_P + FU_BUF;
constexpr int FU_O_ZB = FU_O_Q + FU_BUF;
constexpr int FU_O_W1 = FU_O_ZB + FU_BUF;             // W1 [256][F]
constexpr int FU_O_PAR = FU_O_W1 + HW * kMaxF * 4;    // b1, b2, b3, w4 [256] each; s_in [16]; one
constexpr int FU_O_XQ = FU_O_PAR + (4 * HW + 32) * 4; // x = s_in q [12][F]
constexpr int FU_O_Y = FU_O_XQ + FU_SPT * kMaxF * 4;  // y per point
constexpr int FU_SMEM = FU_O_Y + FU_SPT * 4;
static_assert(FU_SMEM + 1024 <= 227 * 1024, "fused evaluation exceeds shared memory");
static_assert(BM * FU_SCS * 4 <= KT_H * FU_GBLK, "Gram read-out scratch exceeds its region");

template <int F> struct FuCfg {
    static constexpr int R = F + 1;
    static constexpr int NE = F * (F + 1) / 2;
    static constexpr int NJ = F / 2 + 1;                      // partners per direction
    static constexpr int NG = (FU_SPT * F + 15) / 16 * 16;    // Gram N (multiple of 16)
    static_assert(FU_SPT * R <= BM, "points of a tile exceed 128 rows");
    static_assert(NG <= FU_NG, "Gram operand exceeds its region");
};

// Instruction descriptor, kind::f16: FP16 x FP16 -> FP32, both operands K-major.
constexpr uint32_t idesc_f16(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void named_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

// silu and its first two derivatives (fast exponential and division: the
// results feed BF16/FP16 operands)
__device__ __forceinline__ void silu3f(float z, float &f, float &f1, float &f2)
{
    const float s = __fdividef(1.0f, 1.0f + __expf(-fmaxf(z, -80.0f)));
    f = z * s;
    f1 = s * (1.0f + z * (1.0f - s));
    f2 = s * (1.0f - s) * (2.0f + z * (1.0f - 2.0f * s));
}

// Row r (of a canonical K-major operand whose 32-k blocks are blk bytes apart),
// k = 32 ch .. 32 ch + 31, as BF16 or FP16.
template <bool HALF>
__device__ __forceinline__ void put_row32(uint8_t *base, int blk, int r, int ch, const float (&v)[32])
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t h[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if constexpr (HALF) {
                const __half2 x = __floats2half2_rn(v[8 * j + 2 * i], v[8 * j + 2 * i + 1]);
                h[i] = *reinterpret_cast<const uint32_t *>(&x);
            } else {
                const __nv_bfloat162 x = __floats2bfloat162_rn(v[8 * j + 2 * i], v[8 * j + 2 * i + 1]);
                h[i] = *reinterpret_cast<const uint32_t *>(&x);
            }
        }
        *reinterpret_cast<uint4 *>(base + ch * blk + canon_off(r, 8 * j)) = make_uint4(h[0], h[1], h[2], h[3]);
    }
}

__device__ __forceinline__ void put_f32x32(float *dst, const float (&v)[32])
{
#pragma unroll
    for (int i = 0; i < 32; i += 4) *reinterpret_cast<float4 *>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
}

template <int F>
__global__ void __launch_bounds__(320, 1)
    k_mlp_fused(MlpDev m, int64_t n, int n_tiles, const float *__restrict__ q, float *__restrict__ Vout,
                float *__restrict__ gout, float *__restrict__ Hout)
{
    using C = FuCfg<F>;
    constexpr int R = C::R, NE = C::NE, NJ = C::NJ, NG = C::NG, SPT = FU_SPT, PS = FU_PS;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t *sm = smem_raw;
    uint8_t *sA = sm + FU_O_A;
    uint8_t *sB = sm + FU_O_B;
    uint8_t *sG = sm + FU_O_G;
    float *sc = reinterpret_cast<float *>(sm + FU_O_G);      // Gram read-out scratch [128][FU_SCS]
    float *pb = reinterpret_cast<float *>(sm + FU_O_P);      // silu'(z1), silu'(z2), abar2, abar1 -> d1
    float *qb = reinterpret_cast<float *>(sm + FU_O_Q);      // c3, c2, c1, then the layer-1 Hessian terms
    float *zb = reinterpret_cast<float *>(sm + FU_O_ZB);     // value-row staging: a1, a2, delta3, delta2
    float *w1s = reinterpret_cast<float *>(sm + FU_O_W1);
    float *b1s = reinterpret_cast<float *>(sm + FU_O_PAR);
    float *b2s = b1s + HW, *b3s = b2s + HW, *w4s = b3s + HW, *sins = w4s + HW, *one = sins + 16;
    float *xq = reinterpret_cast<float *>(sm + FU_O_XQ);
    float *ys = reinterpret_cast<float *>(sm + FU_O_Y);
    __shared__ uint64_t full_bar[FU_STAGES], empty_bar[FU_STAGES], a_bar, c_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < FU_STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        mbar_init(&a_bar, FU_NC);
        mbar_init(&c_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < HW * F; i += blockDim.x) w1s[i] = m.W1[i];
    for (int i = threadIdx.x; i < HW; i += blockDim.x) {
        b1s[i] = m.b1[i];
        b2s[i] = m.b2[i];
        b3s[i] = m.b3[i];
        w4s[i] = m.w4[i];
    }
    if (threadIdx.x < 16) sins[threadIdx.x] = threadIdx.x < F ? m.s_in[threadIdx.x] : 0.0f;
    if (threadIdx.x == 0) one[0] = 1.0f;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 8) {
        // ---------------- weight producer: per tile W2, W3 (forward), W3^T, W2^T (reverse)
        if (lane == 0) {
            int kc = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x)
                for (int gm = 0; gm < 4 && ok; ++gm) {
                    const uint8_t *Bsrc = gm == 0 ? m.W2t : gm == 1 ? m.W3t : gm == 2 ? m.W3Tt : m.W2Tt;
                    for (int kt = 0; kt < KT_H; ++kt, ++kc) {
                        const int s = kc % FU_STAGES, use = kc / FU_STAGES;
                        if ((use > 0 && !mbar_wait(&empty_bar[s], (use - 1) & 1, kWaitLimitCycles)) ||
                            *(volatile int *)&abort_flag) {
                            atomicExch(&abort_flag, 1);
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&full_bar[s], TILE_B);
                        bulk_g2s(sB + s * TILE_B, Bsrc + (size_t)kt * TILE_B, TILE_B, &full_bar[s]);
                    }
                }
            // do not leave with copies still landing in shared memory
            for (int k = kc - FU_STAGES > 0 ? kc - FU_STAGES : 0; k < kc; ++k)
                mbar_wait(&full_bar[k % FU_STAGES], (k / FU_STAGES) & 1, kWaitLimitCycles);
        }
    } else if (warp == 9) {
        // ---------------- MMA issuer: per tile weight, weight, Gram, weight, Gram, weight
        if (lane == 0) {
            constexpr uint32_t idesc_w = idesc_bf16(BM, BN);
            constexpr uint32_t idesc_g = idesc_f16(BM, NG);
            const uint32_t a0 = su32(sA), b0 = su32(sB), g0 = su32(sG);
            int kc = 0, ca = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x)
                for (int op = 0; op < 6 && ok; ++op) {
                    if (!mbar_wait(&a_bar, ca & 1, kWaitLimitCycles) || *(volatile int *)&abort_flag) {
                        atomicExch(&abort_flag, 1);
                        ok = false;
                        break;
                    }
                    ++ca;
                    tc_fence_after();
                    const uint32_t d = tmem + (op == 0 ? 0u : 256u);
                    if (op == 2 || op == 4) {
                        // Gram product: operands written by the compute warps
#pragma unroll 1
                        for (int kt = 0; kt < KT_H; ++kt)
#pragma unroll
                            for (int ks = 0; ks < BK / 16; ++ks)
                                umma(d, sdesc(a0 + kt * TILE_A + ks * 2 * LBO), sdesc(g0 + kt * FU_GBLK + ks * 2 * LBO),
                                     idesc_g, (kt | ks) != 0);
                    } else {
                        for (int kt = 0; kt < KT_H; ++kt, ++kc) {
                            const int s = kc % FU_STAGES;
                            if (!mbar_wait(&full_bar[s], (kc / FU_STAGES) & 1, kWaitLimitCycles)) {
                                atomicExch(&abort_flag, 1);
                                ok = false;
                                break;
                            }
                            tc_fence_after();
#pragma unroll
                            for (int ks = 0; ks < BK / 16; ++ks)
                                umma(d, sdesc(a0 + kt * TILE_A + ks * 2 * LBO), sdesc(b0 + s * TILE_B + ks * 2 * LBO),
                                     idesc_w, (kt | ks) != 0);
                            umma_commit(&empty_bar[s]);
                        }
                    }
                    umma_commit(&c_bar);   // also on abort: the compute warps are waiting on it
                }
        }
    } else {
        // ---------------- compute warps
        const int c = threadIdx.x;            // 0..255
        const int hf = warp >> 2;             // column half
        const int qd = warp & 3;              // TMEM lane quadrant
        const int r = qd * 32 + lane;         // tile row = TMEM lane
        const int sr = r / R, kr = r % R;     // point of the row; 0 = value row, k = direction k - 1
        const uint32_t lane_base = tmem + ((uint32_t)(qd * 32) << 16);
        const uint32_t col_half = hf * 128;
        // Gram read-out window of quadrant qq: 64 columns from gwin(qq) cover the blocks of
        // every point with a row in it (checked for F = 1..9)
        auto gwin = [](int qq) { return ((qq * 32) / R * F) / 32 * 32; };
        const int gbase = gwin(qd);
        int cc = 0;
        // wait for the accumulator of the current product; uniform outcome over the compute threads
        auto wait_acc = [&]() -> bool {
            if (!mbar_wait(&c_bar, cc & 1, kWaitLimitCycles)) atomicExch(&abort_flag, 1);
            ++cc;
            tc_fence_after();
            named_sync();
            return *(volatile int *)&abort_flag == 0;
        };
        auto release_a = [&]() {
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(&a_bar);
        };
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
            const int64_t p0 = (int64_t)t * SPT;
            const bool valid = sr < SPT && p0 + sr < n;
            const bool prim = valid && kr == 0, tang = valid && kr > 0;
            const int d = tang ? kr - 1 : 0;          // this row's direction
            const float sv = valid ? 1.0f : 0.0f, pv = prim ? 1.0f : 0.0f, tv = tang ? 1.0f : 0.0f;
            const int rowp = (valid ? sr : 0) * PS;   // this row's point in the per-point buffers
            const int gb = (valid ? sr : 0) * F + d;  // this tangent row in the Gram B operand
            float hacc[NJ];
#pragma unroll
            for (int j = 0; j < NJ; ++j) hacc[j] = 0.0f;

            // the read-out of a Gram product (TMEM[256:256+NG)) into hacc, symmetrised
            auto gram_readout = [&]() {
                if (hf == 0) {   // warp-uniform: the first column half reads, the second waits
                    float va[32], vb[32];
                    tmem_ld32(lane_base + 256 + gbase, va);
                    tmem_ld32(lane_base + 256 + gbase + 32, vb);
                    tmem_wait_ld();
                    put_f32x32(sc + r * FU_SCS, va);
                    put_f32x32(sc + r * FU_SCS + 32, vb);
                }
                tc_fence_before();
                named_sync();
                if (tang && hf == 0) {
                    const int c0 = sr * F - gbase;
#pragma unroll
                    for (int j = 0; j < NJ; ++j) {
                        int k = d + j;
                        k = k >= F ? k - F : k;
                        const int rk = sr * R + 1 + k;                 // the partner's row (maybe another quadrant)
                        const float gdk = sc[r * FU_SCS + c0 + k];
                        const float gkd = sc[rk * FU_SCS + sr * F - gwin(rk >> 5) + d];
                        hacc[j] += 0.5f * (gdk + gkd);
                    }
                }
                named_sync();
            };

            // ---- layer 1 (CUDA cores)
            if (c < SPT * F) {
                const int s = c / F, k = c % F;
                const int64_t b = p0 + s;
                xq[c] = b < n ? sins[k] * q[b * F + k] : 0.0f;
            }
            if (c < SPT) ys[c] = *m.b4;
            named_sync();
#pragma unroll 3
            for (int idx = c; idx < SPT * HW; idx += FU_NC) {
                const int s = idx >> 8, o = idx & (HW - 1);
                float z = b1s[o];
#pragma unroll
                for (int k = 0; k < F; ++k) z = fmaf(w1s[o * F + k], xq[s * F + k], z);
                float f, f1, f2;
                silu3f(z, f, f1, f2);
                zb[s * PS + o] = f;
                pb[s * PS + o] = f1;
            }
            named_sync();
            {
                const float *src = (prim ? zb : pb) + rowp;
                const float *fac = tang ? w1s + d : one;
                const int fst = tang ? F : 0;
#pragma unroll 1
                for (int j = 0; j < 4; ++j) {
                    const int ch = hf * 4 + j;
                    float v[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int o = ch * 32 + i;
                        v[i] = sv * src[o] * fac[o * fst];
                    }
                    put_row32<false>(sA, TILE_A, r, ch, v);
                }
            }
            release_a();

            // ---- layer 2: TMEM[0:256) holds z2 - b2 (value rows) and J2 (tangent rows)
            if (!wait_acc()) break;
#pragma unroll 1
            for (int j = 0; j < 4; j += 2) {
                float v[32], u[32];
                tmem_ld32(lane_base + col_half + j * 32, v);
                tmem_ld32(lane_base + col_half + (j + 1) * 32, u);
                tmem_wait_ld();
                if (prim) {
                    put_f32x32(zb + rowp + (hf * 4 + j) * 32, v);
                    put_f32x32(zb + rowp + (hf * 4 + j + 1) * 32, u);
                }
            }
            named_sync();
#pragma unroll 3
            for (int idx = c; idx < SPT * HW; idx += FU_NC) {
                const int s = idx >> 8, o = idx & (HW - 1);
                float f, f1, f2;
                silu3f(zb[s * PS + o] + b2s[o], f, f1, f2);
                zb[s * PS + o] = f;
                pb[s * PS + o] = f1;
            }
            named_sync();
            {
                const float *src = (prim ? zb : pb) + rowp;
#pragma unroll 1
                for (int j = 0; j < 4; j += 2) {
                    float v[32], u[32];
                    tmem_ld32(lane_base + col_half + j * 32, v);
                    tmem_ld32(lane_base + col_half + (j + 1) * 32, u);
                    tmem_wait_ld();
                    const int ch = hf * 4 + j;
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] = sv * src[ch * 32 + i] * fmaf(pv, 1.0f - v[i], v[i]);
                    put_row32<false>(sA, TILE_A, r, ch, v);
#pragma unroll
                    for (int i = 0; i < 32; ++i) u[i] = sv * src[ch * 32 + 32 + i] * fmaf(pv, 1.0f - u[i], u[i]);
                    put_row32<false>(sA, TILE_A, r, ch + 1, u);
                }
            }
            release_a();

            // ---- layer 3: TMEM[256:512) holds z3 - b3 and J3; V, delta3, c3 and the Gram operands
            if (!wait_acc()) break;
#pragma unroll 1
            for (int j = 0; j < 4; j += 2) {
                float v[32], u[32];
                tmem_ld32(lane_base + 256 + col_half + j * 32, v);
                tmem_ld32(lane_base + 256 + col_half + (j + 1) * 32, u);
                tmem_wait_ld();
                if (prim) {
                    put_f32x32(zb + rowp + (hf * 4 + j) * 32, v);
                    put_f32x32(zb + rowp + (hf * 4 + j + 1) * 32, u);
                }
            }
            named_sync();
#pragma unroll 3
            for (int idx = c; idx < SPT * HW; idx += FU_NC) {   // the 256 entries of one pass share a point
                const int s = idx >> 8, o = idx & (HW - 1);
                float f, f1, f2;
                silu3f(zb[s * PS + o] + b3s[o], f, f1, f2);
                const float w4 = w4s[o];
                zb[s * PS + o] = w4 * f1;        // delta3
                qb[s * PS + o] = w4 * f2;        // c3
                float y = w4 * f;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) y += __shfl_xor_sync(0xffffffffu, y, off);
                if (lane == 0) atomicAdd(&ys[s], y);
            }
            named_sync();
            if (prim && hf == 0) Vout[p0 + sr] = m.s_out * ys[sr];
#pragma unroll 1
            for (int j = 0; j < 4; ++j) {                     // Gram operands: c3 J3 (A), J3 (B, tangent rows)
                const int ch = hf * 4 + j;
                float v[32], w[32];
                tmem_ld32(lane_base + 256 + col_half + j * 32, v);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 32; ++i) w[i] = tv * qb[rowp + ch * 32 + i] * v[i];
                put_row32<true>(sA, TILE_A, r, ch, w);
                if (tang) put_row32<true>(sG, FU_GBLK, gb, ch, v);
            }
            release_a();
            if (!wait_acc()) break;                           // Gram product of layer 3 done
            gram_readout();
#pragma unroll 1
            for (int j = 0; j < 4; ++j) {                     // delta3 rows
                const int ch = hf * 4 + j;
                float x[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) x[i] = pv * zb[rowp + ch * 32 + i];
                put_row32<false>(sA, TILE_A, r, ch, x);
            }
            release_a();

            // ---- reverse through layer 3: TMEM[256:512) = abar2 (value rows); TMEM[0:256) = z2 - b2, J2
            if (!wait_acc()) break;
#pragma unroll 1
            for (int j = 0; j < 4; ++j) {
                float v[32], u[32];
                tmem_ld32(lane_base + 256 + col_half + j * 32, v);
                tmem_ld32(lane_base + col_half + j * 32, u);
                tmem_wait_ld();
                if (prim) {
                    put_f32x32(pb + rowp + (hf * 4 + j) * 32, v);
                    put_f32x32(zb + rowp + (hf * 4 + j) * 32, u);
                }
            }
            named_sync();
#pragma unroll 3
            for (int idx = c; idx < SPT * HW; idx += FU_NC) {
                const int s = idx >> 8, o = idx & (HW - 1);
                float f, f1, f2;
                silu3f(zb[s * PS + o] + b2s[o], f, f1, f2);
                const float ab = pb[s * PS + o];
                zb[s * PS + o] = ab * f1;        // delta2 = abar2 silu'(z2)
                qb[s * PS + o] = ab * f2;        // c2 = abar2 silu''(z2)
            }
            named_sync();
#pragma unroll 1
            for (int j = 0; j < 4; ++j) {                     // Gram operands: c2 J2 (A), J2 (B)
                const int ch = hf * 4 + j;
                float v[32], w[32];
                tmem_ld32(lane_base + col_half + j * 32, v);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 32; ++i) w[i] = tv * qb[rowp + ch * 32 + i] * v[i];
                put_row32<true>(sA, TILE_A, r, ch, w);
                if (tang) put_row32<true>(sG, FU_GBLK, gb, ch, v);
            }
            release_a();
            if (!wait_acc()) break;                           // Gram product of layer 2 done
            gram_readout();
#pragma unroll 1
            for (int j = 0; j < 4; ++j) {                     // delta2 rows
                const int ch = hf * 4 + j;
                float x[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) x[i] = pv * zb[rowp + ch * 32 + i];
                put_row32<false>(sA, TILE_A, r, ch, x);
            }
            release_a();

            // ---- reverse through layer 2: TMEM[256:512) = abar1; grad V and the layer-1 term
            if (!wait_acc()) break;
#pragma unroll 1
            for (int j = 0; j < 4; j += 2) {
                float v[32], u[32];
                tmem_ld32(lane_base + 256 + col_half + j * 32, v);
                tmem_ld32(lane_base + 256 + col_half + (j + 1) * 32, u);
                tmem_wait_ld();
                if (prim) {
                    put_f32x32(pb + rowp + (hf * 4 + j) * 32, v);
                    put_f32x32(pb + rowp + (hf * 4 + j + 1) * 32, u);
                }
            }
            tc_fence_before();
            named_sync();
#pragma unroll 3
            for (int idx = c; idx < SPT * HW; idx += FU_NC) {
                const int s = idx >> 8, o = idx & (HW - 1);
                float z = b1s[o];
#pragma unroll
                for (int k = 0; k < F; ++k) z = fmaf(w1s[o * F + k], xq[s * F + k], z);
                float f, f1, f2;
                silu3f(z, f, f1, f2);
                const float ab = pb[s * PS + o];
                pb[s * PS + o] = ab * f1;        // d1 = abar1 silu'(z1)
                qb[s * PS + o] = ab * f2;        // c1 = abar1 silu''(z1)
            }
            named_sync();
            // grad V and H1 = W1^T diag(c1) W1: thread (point s, slice sl) sums 16 hidden units,
            // then the 16 slices of a point (adjacent lanes) are added by shuffles
            if (c < SPT * 16) {
                const int s = c >> 4, sl = c & 15;
                float ga[F], ha[NE];
#pragma unroll
                for (int k = 0; k < F; ++k) ga[k] = 0.0f;
#pragma unroll
                for (int e = 0; e < NE; ++e) ha[e] = 0.0f;
#pragma unroll 1
                for (int oo = 0; oo < 16; ++oo) {
                    const int o = sl * 16 + ((oo + sl) & 15);   // staggered start: fewer bank conflicts
                    const float d1 = pb[s * PS + o], c1 = qb[s * PS + o];
                    float wk[F];
#pragma unroll
                    for (int k = 0; k < F; ++k) wk[k] = w1s[o * F + k];
                    int e = 0;
#pragma unroll
                    for (int k1 = 0; k1 < F; ++k1) {
                        ga[k1] = fmaf(d1, wk[k1], ga[k1]);
                        const float cw = c1 * wk[k1];
#pragma unroll
                        for (int k2 = k1; k2 < F; ++k2, ++e) ha[e] = fmaf(cw, wk[k2], ha[e]);
                    }
                }
#pragma unroll
                for (int off = 1; off < 16; off <<= 1) {
#pragma unroll
                    for (int k = 0; k < F; ++k) ga[k] += __shfl_xor_sync(0xffffffffu, ga[k], off);
#pragma unroll
                    for (int e = 0; e < NE; ++e) ha[e] += __shfl_xor_sync(0xffffffffu, ha[e], off);
                }
                const int64_t b = p0 + s;
                if (sl == 0 && b < n) {
#pragma unroll
                    for (int k = 0; k < F; ++k) gout[b * F + k] = m.s_out * sins[k] * ga[k];
                }
                if (sl == 0) {
#pragma unroll
                    for (int e = 0; e < NE; ++e) zb[s * PS + e] = ha[e];
                }
            }
            named_sync();
            if (tang && hf == 0) {
                const int64_t b = p0 + sr;
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    int k = d + j;
                    k = k >= F ? k - F : k;
                    if ((F % 2 == 0) && j == F / 2 && d >= F / 2) continue;   // pair already taken
                    const int lo = d < k ? d : k, hi = d < k ? k : d;
                    const int e = lo * F - lo * (lo - 1) / 2 + (hi - lo);
                    const float h = m.s_out * sins[d] * sins[k] * (hacc[j] + zb[rowp + e]);
                    Hout[(b * F + d) * F + k] = h;
                    Hout[(b * F + k) * F + d] = h;
                }
            }
            named_sync();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// ---------------------------------------------------------------- host side
inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct EvalLayout {
    int spt, R;
    int64_t n_tiles, M_pad, n_pad;
    size_t X2, X3, D3, D2, Z1, C2, C3, Ab2, Ab1, total;
};

inline EvalLayout eval_layout(int F, int64_t n, bool hess)
{
    EvalLayout L{};
    L.R = hess ? F + 1 : 1;
    L.spt = BM / L.R;
    L.n_tiles = (n + L.spt - 1) / L.spt;
    L.M_pad = L.n_tiles * BM;
    L.n_pad = (n + BM - 1) / BM * BM;
    size_t o = 0;
    L.X2 = o; o += a256((size_t)L.M_pad * HW * 2);
    L.X3 = o; o += a256((size_t)L.M_pad * HW * 2);
    L.D3 = o; o += a256((size_t)L.n_pad * HW * 2);
    L.D2 = o; o += a256((size_t)L.n_pad * HW * 2);
    L.Z1 = o; o += a256((size_t)L.n_pad * HW * 4);
    L.C2 = o; o += a256((size_t)L.M_pad * HW * 4);
    L.C3 = o; o += a256((size_t)L.M_pad * HW * 4);
    L.Ab2 = o; o += a256((size_t)L.n_pad * HW * 4);
    L.Ab1 = o; o += a256((size_t)L.n_pad * HW * 4);
    L.total = o;
    return L;
}

struct TrainLayout {
    int64_t n_tiles, M_pad;
    int n_kt_rows, n_split, kt_split;
    size_t V1, g1, X2, X3, D3, D2, X2T, X3T, D3T, D2T, C2, C3, Ab2, Ab1, Z1, Zd1, X0, Xd0, ebar, part, GW2, GW3, eval,
        total;
};

inline TrainLayout train_layout(int F, int64_t n)
{
    TrainLayout L{};
    L.n_tiles = (n + TR_SPT - 1) / TR_SPT;
    L.M_pad = L.n_tiles * BM;
    L.n_kt_rows = (int)(L.M_pad / BK);
    L.n_split = L.n_kt_rows < 74 ? L.n_kt_rows : 74;   // 2 x 74 CTAs for the weight-gradient GEMMs
    L.kt_split = (L.n_kt_rows + L.n_split - 1) / L.n_split;
    L.n_split = (L.n_kt_rows + L.kt_split - 1) / L.kt_split;
    const size_t tb = a256((size_t)L.M_pad * HW * 2), tf = a256((size_t)L.M_pad * HW * 4);
    const size_t nf = a256((size_t)n * HW * 4);
    size_t o = 0;
    L.V1 = o; o += a256((size_t)n * 4);
    L.g1 = o; o += a256((size_t)n * F * 4);
    L.X2 = o; o += tb;
    L.X3 = o; o += tb;
    L.D3 = o; o += tb;
    L.D2 = o; o += tb;
    L.X2T = o; o += tb;
    L.X3T = o; o += tb;
    L.D3T = o; o += tb;
    L.D2T = o; o += tb;
    L.C2 = o; o += tf;
    L.C3 = o; o += tf;
    L.Ab2 = o; o += tf;
    L.Ab1 = o; o += tf;
    L.Z1 = o; o += nf;
    L.Zd1 = o; o += nf;
    L.X0 = o; o += a256((size_t)n * F * 4);
    L.Xd0 = o; o += a256((size_t)n * F * 4);
    L.ebar = o; o += a256((size_t)n * 4);
    L.part = o; o += a256((size_t)L.n_tiles * part_len(F) * 4);
    L.GW2 = o; o += a256((size_t)L.n_split * HW * HW * 4);
    L.GW3 = o; o += a256((size_t)L.n_split * HW * HW * 4);
    L.eval = o; o += eval_layout(F, n, false).total;
    L.total = o;
    return L;
}

MlpDev make_dev(const MlpWeightsDev &w, int F, int R)
{
    MlpDev m{};
    m.F = F;
    m.rows_per_sample = R;
    m.spt = BM / R;
    m.W1 = w.W1; m.b1 = w.b1; m.W2 = w.W2; m.b2 = w.b2; m.W3 = w.W3; m.b3 = w.b3; m.w4 = w.w4;
    m.b4 = w.b4; m.s_out = w.s_out; m.s_in = w.s_in;
    m.W2t = w.W2t; m.W3t = w.W3t; m.W2Tt = w.W2Tt; m.W3Tt = w.W3Tt;
    return m;
}

cudaError_t set_smem_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_layer1, cudaFuncAttributeMaxDynamicSharedMemorySize, BM * HW * 4);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_hidden_act, cudaFuncAttributeMaxDynamicSharedMemorySize, TSMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tr_layer1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TSMEM + 2 * TR_SPT * kMaxF * 4);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tr_out, cudaFuncAttributeMaxDynamicSharedMemorySize, TSMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tr_back, cudaFuncAttributeMaxDynamicSharedMemorySize, TSMEM);
#define SCIVR_FA(FF) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_fused<FF>, cudaFuncAttributeMaxDynamicSharedMemorySize, FU_SMEM);
    SCIVR_FA(1) SCIVR_FA(2) SCIVR_FA(3) SCIVR_FA(4) SCIVR_FA(5) SCIVR_FA(6) SCIVR_FA(7) SCIVR_FA(8) SCIVR_FA(9)
#undef SCIVR_FA
    return e;
}

// Forward GEMM over a whole row-tiled operand (K = 256, N = 256).
inline void gemm_rows(const uint8_t *A, const uint8_t *B, float *C, int64_t rows, cudaStream_t s)
{
    k_gemm<<<dim3(1, (unsigned)(rows / BM), 1), 128, GEMM_SMEM, s>>>(A, B, KT_H, KT_H, C, HW, rows, 0);
}

// V and grad V (no Hessian): one row per point through the unfused kernels
// (layer 1, two GEMMs with activation, output, two reverse GEMMs, gradient).
template <int F>
cudaError_t eval_F(const MlpWeightsDev &w, int64_t n, const float *q, float *V, float *g, uint8_t *scr,
                   cudaStream_t s, int *n_launch)
{
    const EvalLayout L = eval_layout(F, n, false);
    const MlpDev m = make_dev(w, F, L.R);
    uint8_t *X2 = scr + L.X2, *X3 = scr + L.X3, *D3 = scr + L.D3, *D2 = scr + L.D2;
    float *Z1 = reinterpret_cast<float *>(scr + L.Z1), *C2 = reinterpret_cast<float *>(scr + L.C2);
    float *C3 = reinterpret_cast<float *>(scr + L.C3), *Ab2 = reinterpret_cast<float *>(scr + L.Ab2);
    float *Ab1 = reinterpret_cast<float *>(scr + L.Ab1);
    const unsigned nt = (unsigned)L.n_tiles;
    k_layer1<<<nt, 256, (size_t)L.spt * HW * 4, s>>>(m, n, q, X2, Z1);
    gemm_rows(X2, m.W2t, C2, L.M_pad, s);
    k_hidden_act<<<nt, 256, TSMEM, s>>>(m, n, C2, m.b2, X3, nullptr, 0);
    gemm_rows(X3, m.W3t, C3, L.M_pad, s);
    k_output<<<(unsigned)L.n_pad, 256, 0, s>>>(m, n, C3, V, D3);
    gemm_rows(D3, m.W3Tt, Ab2, L.n_pad, s);
    const int64_t nbk = L.n_pad * (HW / 8);
    k_backward_act<<<(unsigned)((nbk + 255) / 256), 256, 0, s>>>(m, n, Ab2, C2, m.b2, D2);
    gemm_rows(D2, m.W2Tt, Ab1, L.n_pad, s);
    k_grad<F><<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(m, n, Z1, Ab1, g);
    *n_launch = 9;
    return cudaGetLastError();
}

template <int F>
cudaError_t eval_fused_F(const MlpWeightsDev &w, int64_t n, const float *q, float *V, float *g, float *H,
                         cudaStream_t s, int *n_launch)
{
    const MlpDev m = make_dev(w, F, F + 1);
    const int64_t n_tiles = (n + FU_SPT - 1) / FU_SPT;
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = (int)(n_tiles < n_sm ? n_tiles : n_sm);
    k_mlp_fused<F><<<grid, 320, FU_SMEM, s>>>(m, n, (int)n_tiles, q, V, g, H);
    *n_launch = 1;
    return cudaGetLastError();
}

template <int F>
cudaError_t loss_grad_F(const MlpWeightsDev &w, int64_t n, const float *q, const float *Vref, const float *gref,
                        float alpha, float beta, float *grad, float *loss, uint8_t *scr, cudaStream_t s,
                        int *n_launch)
{
    const TrainLayout L = train_layout(F, n);
    auto fp = [&](size_t off) { return reinterpret_cast<float *>(scr + off); };
    float *V1 = fp(L.V1), *g1 = fp(L.g1);
    int nl = 0;
    cudaError_t e = eval_F<F>(w, n, q, V1, g1, scr + L.eval, s, &nl);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    const MlpDev m = make_dev(w, F, 2);
    const unsigned nt = (unsigned)L.n_tiles;
    uint8_t *X2 = scr + L.X2, *X3 = scr + L.X3, *D3 = scr + L.D3, *D2 = scr + L.D2;
    uint8_t *X2T = scr + L.X2T, *X3T = scr + L.X3T, *D3T = scr + L.D3T, *D2T = scr + L.D2T;
    float *C2 = fp(L.C2), *C3 = fp(L.C3), *Ab2 = fp(L.Ab2), *Ab1 = fp(L.Ab1), *part = fp(L.part);
    k_tr_layer1<<<nt, 256, TSMEM + 2 * TR_SPT * kMaxF * 4, s>>>(m, n, q, V1, g1, Vref, gref, alpha, beta,
                                                               1.0f / (float)n, X2, X2T, L.n_kt_rows, fp(L.Z1),
                                                               fp(L.Zd1), fp(L.X0), fp(L.Xd0), fp(L.ebar), loss);
    gemm_rows(X2, m.W2t, C2, L.M_pad, s);
    k_hidden_act<<<nt, 256, TSMEM, s>>>(m, n, C2, m.b2, X3, X3T, L.n_kt_rows);
    gemm_rows(X3, m.W3t, C3, L.M_pad, s);
    k_tr_out<<<nt, 256, TSMEM, s>>>(m, n, C3, fp(L.ebar), D3, D3T, L.n_kt_rows, part);
    gemm_rows(D3, m.W3Tt, Ab2, L.M_pad, s);
    k_tr_back<<<nt, 256, TSMEM, s>>>(m, n, Ab2, C2, D2, D2T, L.n_kt_rows, part);
    gemm_rows(D2, m.W2Tt, Ab1, L.M_pad, s);
    k_tr_back1<F><<<nt, 256, 0, s>>>(m, n, Ab1, fp(L.Z1), fp(L.Zd1), fp(L.X0), fp(L.Xd0), part);
    // weight gradients of the 256 x 256 layers: [out][in] = sum over rows of D^T X
    const dim3 gw(1, HW / BM, (unsigned)L.n_split);
    k_gemm<<<gw, 128, GEMM_SMEM, s>>>(D2T, X2T, L.n_kt_rows, L.kt_split, fp(L.GW2), HW, HW, (int64_t)HW * HW);
    k_gemm<<<gw, 128, GEMM_SMEM, s>>>(D3T, X3T, L.n_kt_rows, L.kt_split, fp(L.GW3), HW, HW, (int64_t)HW * HW);
    const int64_t n_par = (int64_t)HW * F + 2 * HW * HW + 4 * HW + 1;
    k_tr_reduce<<<(unsigned)((n_par + 255) / 256), 256, 0, s>>>(F, (int)L.n_tiles, part, L.n_split, fp(L.GW2),
                                                               fp(L.GW3), grad);
    *n_launch = nl + 12;
    return cudaGetLastError();
}

}  // namespace mlp

size_t mlp_eval_scratch_bytes(int F, int64_t n, bool hess)
{
    return hess ? 256 : mlp::eval_layout(F, n, false).total;   // the Hessian path keeps everything on chip
}
size_t mlp_train_scratch_bytes(int F, int64_t n) { return mlp::train_layout(F, n).total; }

cudaError_t mlp_prepare() { return mlp::set_smem_attributes(); }

cudaError_t mlp_eval(const MlpWeightsDev &w, int F, int64_t n, const float *q, float *V, float *g, float *H,
                     void *scratch, cudaStream_t s, int *n_launch)
{
    uint8_t *scr = static_cast<uint8_t *>(scratch);
    switch (F) {
#define SCIVR_M(FF)                                                                         \
    case FF:                                                                                \
        return H ? mlp::eval_fused_F<FF>(w, n, q, V, g, H, s, n_launch)                     \
                 : mlp::eval_F<FF>(w, n, q, V, g, scr, s, n_launch);
    SCIVR_M(1) SCIVR_M(2) SCIVR_M(3) SCIVR_M(4) SCIVR_M(5) SCIVR_M(6) SCIVR_M(7) SCIVR_M(8) SCIVR_M(9)
#undef SCIVR_M
    default: *n_launch = 0; return cudaErrorInvalidValue;
    }
}

cudaError_t mlp_loss_grad(const MlpWeightsDev &w, int F, int64_t n, const float *q, const float *Vref,
                          const float *gref, float alpha, float beta, float *grad, float *loss, void *scratch,
                          cudaStream_t s, int *n_launch)
{
    uint8_t *scr = static_cast<uint8_t *>(scratch);
    switch (F) {
#define SCIVR_M(FF) case FF: return mlp::loss_grad_F<FF>(w, n, q, Vref, gref, alpha, beta, grad, loss, scr, s, n_launch);
    SCIVR_M(1) SCIVR_M(2) SCIVR_M(3) SCIVR_M(4) SCIVR_M(5) SCIVR_M(6) SCIVR_M(7) SCIVR_M(8) SCIVR_M(9)
#undef SCIVR_M
    default: *n_launch = 0; return cudaErrorInvalidValue;
    }
}

cudaError_t mlp_tile_weights(const MlpWeightsDev &w, cudaStream_t s)
{
    const int n = mlp::HW * (mlp::HW / 8);
    mlp::k_tile_weight<<<(n + 255) / 256, 256, 0, s>>>(w.W2, 0, w.W2t);
    mlp::k_tile_weight<<<(n + 255) / 256, 256, 0, s>>>(w.W3, 0, w.W3t);
    mlp::k_tile_weight<<<(n + 255) / 256, 256, 0, s>>>(w.W2, 1, w.W2Tt);
    mlp::k_tile_weight<<<(n + 255) / 256, 256, 0, s>>>(w.W3, 1, w.W3Tt);
    return cudaGetLastError();
}

cudaError_t mlp_adamw(const MlpWeightsDev &w, const float *grad, float *m1, float *m2, float lr, float beta1,
                      float beta2, float eps, float wd, float c1, float c2, cudaStream_t s)
{
    mlp::k_adamw<<<(unsigned)((w.n_params + 255) / 256), 256, 0, s>>>(w.theta, grad, m1, m2, w.n_params, lr, beta1,
                                                                       beta2, eps, wd, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return mlp_tile_weights(w, s);
}

cudaError_t read_and_clear_status_mlp(int *status)
{
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(status, g_device_status, sizeof(int));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_device_status, &zero, sizeof(int));
}

}  // namespace scivr
