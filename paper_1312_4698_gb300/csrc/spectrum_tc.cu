// Time -> energy Fourier step (Eq. I(E)_discreto of arXiv:1312.4698) on the
// 5th-generation tensor cores (tcgen05, sm_103a).
//
// The complex contraction X = a . tw (n_traj x K times K x n_E) is written
// as one real GEMM  [Re a | Im a] . [[cos, sin], [-sin, cos]]  with
// M = n_traj, N = 2 n_E (each 256-column tile holds the real parts of 128
// energies followed by their imaginary parts), K' = 2K.  Each FP64/FP32
// operand is split into ND BF16 digits (x ~ d0 + d1 + d2, d_i = bf16 of the
// remainder) and the digit products with d_a + d_b < ND are accumulated in
// one FP32 TMEM accumulator: ND = 1 is plain BF16, ND = 2 keeps ~16 bits
// (3 products), ND = 3 keeps FP32-level accuracy (6 products).
//
// Operands are pre-tiled in HBM in the tensor core's canonical K-major
// no-swizzle layout (8-row x 16-byte core matrices), so each pipeline stage
// is one contiguous bulk copy (cp.async.bulk) per operand.  One CTA per
// 128 x 256 output tile: warp 0 lane 0 issues the copies, warp 1 lane 0
// issues tcgen05.mma from one elected thread, and all four warps read the
// accumulator back with tcgen05.ld and reduce w_j |X_jk|^2 over the tile's
// rows.  Every mbarrier wait is bounded; an expired wait records
// SCIVR_ETIMEOUT in a device status word and the CTA winds down.
#include <cuda_bf16.h>

#include <cstdint>

#include "tc_common.cuh"

namespace scivr {
namespace tc {

template <int ND>
__device__ __forceinline__ void split_digits(float x, __nv_bfloat16 (&d)[ND])
{
    float r = x;
#pragma unroll
    for (int i = 0; i < ND; ++i) {
        d[i] = __float2bfloat16_rn(r);
        r -= __bfloat162float(d[i]);
    }
}

// A' rows: [Re a(0..K-1), Im a(0..K-1), 0 ...]; rows of bad or missing trajectories are zero.
// One thread: one row, one 8-column chunk, all digits.
template <int ND>
__global__ void k_split_amp(const AmpRef amp, int64_t amp_ld, const uint8_t *__restrict__ good,
                            int64_t n_traj, int K, int n_kt, int64_t rows_pad, uint8_t *__restrict__ At)
{
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int chunks = n_kt * (BK / 8);
    if (gid >= rows_pad * chunks) return;
    // row fastest inside groups of 8 so that 8 threads fill one 128-byte core matrix
    const int64_t grp = gid / (8 * (int64_t)chunks);
    const int rem = (int)(gid % (8 * (int64_t)chunks));
    const int ch = rem / 8;
    const int64_t r = grp * 8 + (rem % 8);
    const int k0 = ch * 8;
    const bool ok = r < n_traj && good[r];
    __nv_bfloat16 dg[ND][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int kp = k0 + i;
        float x = 0.0f;
        if (ok) {
            if (kp < K) x = amp.re_f(r * amp_ld + kp);
            else if (kp < 2 * K) x = amp.im_f(r * amp_ld + (kp - K));
        }
        __nv_bfloat16 d[ND];
        split_digits<ND>(x, d);
#pragma unroll
        for (int q = 0; q < ND; ++q) dg[q][i] = d[q];
    }
    const int64_t mt = r / BM;
    const int kt = k0 / BK;
    const uint32_t off = canon_off((int)(r % BM), k0 % BK);
#pragma unroll
    for (int q = 0; q < ND; ++q) {
        uint8_t *dst = At + (((mt * n_kt + kt) * ND + q) * (int64_t)TILE_A) + off;
        *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(&dg[q][0]);
    }
}

// B' rows of tile nt: rows 0..127 are Re rows of energies nt*128 + i, rows 128..255 Im rows.
// Re row: [cos(E c dt), -sin(E c dt)]; Im row: [sin(E c dt), cos(E c dt)].
template <int ND>
__global__ void k_split_tw(int K, int n_kt, int n_E, int n_nt, double E_min, double dE, double dt,
                           uint8_t *__restrict__ Bt)
{
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int chunks = n_kt * (BK / 8);
    const int64_t rows = (int64_t)n_nt * BN;
    if (gid >= rows * chunks) return;
    const int64_t grp = gid / (8 * (int64_t)chunks);
    const int rem = (int)(gid % (8 * (int64_t)chunks));
    const int ch = rem / 8;
    const int64_t n = grp * 8 + (rem % 8);
    const int nt = (int)(n / BN), nr = (int)(n % BN);
    const int e = nt * EPT + (nr % EPT);
    const bool im_row = nr >= EPT;
    const int k0 = ch * 8;
    __nv_bfloat16 dg[ND][8];
    const double E = E_min + e * dE;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int kp = k0 + i;
        float v = 0.0f;
        if (e < n_E && kp < 2 * K) {
            const int c = kp < K ? kp : kp - K;
            const double turns = E * (c * dt) * kInvTwoPi;
            const float fr = (float)(turns - rint(turns));
            float sn, cs;
            sincospif(2.0f * fr, &sn, &cs);
            if (!im_row) v = kp < K ? cs : -sn;
            else v = kp < K ? sn : cs;
        }
        __nv_bfloat16 d[ND];
        split_digits<ND>(v, d);
#pragma unroll
        for (int q = 0; q < ND; ++q) dg[q][i] = d[q];
    }
    const int kt = k0 / BK;
    const uint32_t off = canon_off(nr, k0 % BK);
#pragma unroll
    for (int q = 0; q < ND; ++q) {
        uint8_t *dst = Bt + ((((int64_t)nt * n_kt + kt) * ND + q) * (int64_t)TILE_B) + off;
        *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(&dg[q][0]);
    }
}

template <int ND>
__global__ void __launch_bounds__(128, 1)
    k_ft_tc(const uint8_t *__restrict__ At, const uint8_t *__restrict__ Bt, const double *__restrict__ w,
            const uint8_t *__restrict__ good, int64_t n_traj, int n_kt, int n_E, double *__restrict__ part)
{
    using CF = Cfg<ND>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full_bar[CF::STAGES], empty_bar[CF::STAGES], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nt = blockIdx.x;
    const int64_t mt = blockIdx.y;

    if (threadIdx.x == 0) {
        for (int s = 0; s < CF::STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    const uint8_t *Ablk = At + (size_t)mt * n_kt * CF::A_BYTES;
    const uint8_t *Bblk = Bt + (size_t)nt * n_kt * CF::B_BYTES;

    if (warp == 0 && lane == 0) {
        // producer: one bulk copy per operand per stage
        int issued = 0;
        for (int kt = 0; kt < n_kt; ++kt) {
            const int s = kt % CF::STAGES, use = kt / CF::STAGES;
            if (use > 0 && !mbar_wait(&empty_bar[s], (use - 1) & 1, kWaitLimitCycles)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            if (*(volatile int *)&abort_flag) break;
            uint8_t *sa = smem + s * CF::STAGE;
            uint8_t *sb = sa + CF::A_BYTES;
            mbar_expect_tx(&full_bar[s], CF::A_BYTES + CF::B_BYTES);
            bulk_g2s(sa, Ablk + (size_t)kt * CF::A_BYTES, CF::A_BYTES, &full_bar[s]);
            bulk_g2s(sb, Bblk + (size_t)kt * CF::B_BYTES, CF::B_BYTES, &full_bar[s]);
            issued = kt + 1;
        }
        // never leave with copies in flight: wait (bounded) for the last use of each stage
        for (int kt = issued - CF::STAGES > 0 ? issued - CF::STAGES : 0; kt < issued; ++kt)
            mbar_wait(&full_bar[kt % CF::STAGES], (kt / CF::STAGES) & 1, kWaitLimitCycles);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(BM, BN);
        constexpr int pa[6] = {0, 0, 1, 0, 1, 2};
        constexpr int pb[6] = {0, 1, 0, 2, 1, 0};
        bool ok = true;
        for (int kt = 0; kt < n_kt && ok; ++kt) {
            const int s = kt % CF::STAGES;
            if (!mbar_wait(&full_bar[s], (kt / CF::STAGES) & 1, kWaitLimitCycles) || *(volatile int *)&abort_flag) {
                atomicExch(&abort_flag, 1);
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t sa = su32(smem + s * CF::STAGE);
            const uint32_t sb = sa + CF::A_BYTES;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
#pragma unroll
                for (int p = 0; p < CF::NPAIR; ++p) {
                    const uint64_t ad = sdesc(sa + pa[p] * TILE_A + ks * 2 * LBO);
                    const uint64_t bd = sdesc(sb + pb[p] * TILE_B + ks * 2 * LBO);
                    umma(tmem, ad, bd, idesc, (kt | ks | p) != 0);
                }
            }
            umma_commit(&empty_bar[s]);
        }
        umma_commit(&done_bar);
    }
    __syncwarp();
    // epilogue: all 128 threads, row = 32 * warp + lane
    const bool done_ok = mbar_wait(&done_bar, 0, kWaitLimitCycles) && !*(volatile int *)&abort_flag;
    tc_fence_after();
    __syncwarp();
    float *stg = reinterpret_cast<float *>(smem);   // [BM][EPT + 1], reuses the stage buffers
    const int row = warp * 32 + lane;
    const int64_t grow = mt * BM + row;
    const bool ok = done_ok && grow < n_traj && good[grow];
    const float wr = ok ? (float)w[grow] : 0.0f;
#pragma unroll 1
    for (int ch = 0; ch < EPT / 32; ++ch) {
        float re[32], im[32];
        const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16);
        tmem_ld32(base + ch * 32, re);
        tmem_ld32(base + EPT + ch * 32, im);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const float m2 = fmaf(re[i], re[i], im[i] * im[i]);
            stg[row * (EPT + 1) + ch * 32 + i] = ok ? wr * m2 : 0.0f;
        }
    }
    tc_fence_before();
    __syncthreads();
    {
        const int e = nt * EPT + threadIdx.x;
        double s = 0.0;
#pragma unroll 8
        for (int r = 0; r < BM; ++r) s += (double)stg[r * (EPT + 1) + threadIdx.x];
        if (e < n_E) part[mt * n_E + e] = s;
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
    }
}

__global__ void k_tc_count_good(const uint8_t *__restrict__ good, int64_t n, int64_t *__restrict__ out,
                                int64_t *__restrict__ out2)
{
    __shared__ long long red[1024];
    long long acc = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += good[i] ? 1 : 0;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = red[0];
        if (out2) out2[0] = red[0];
    }
}

__global__ void k_tc_reduce(const double *__restrict__ part, int n_mt, int n_E, const int64_t *__restrict__ ng,
                            double scale, double *__restrict__ I_out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_E) return;
    double s = 0.0;
    for (int m = 0; m < n_mt; ++m) s += part[(int64_t)m * n_E + k];
    I_out[k] = ng[0] > 0 ? s * (scale / (double)ng[0]) : 0.0;
}

// Waits on an mbarrier that nothing completes, with a short limit: the
// bounded-wait path must set SCIVR_ETIMEOUT and return.
__global__ void k_wait_selftest(long long limit)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0, limit);
}

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct TcLayout {
    int K, n_kt, n_nt;
    int64_t n_mt, rows_pad;
    size_t off_ng, off_part, off_A, off_B, total;
};

inline TcLayout tc_layout(int nd, int64_t n_traj, int n_steps, int n_E)
{
    TcLayout L{};
    L.K = n_steps + 1;
    L.n_kt = (2 * L.K + BK - 1) / BK;
    L.n_mt = (n_traj + BM - 1) / BM;
    L.rows_pad = L.n_mt * BM;
    L.n_nt = (n_E + EPT - 1) / EPT;
    L.off_ng = 0;
    L.off_part = a256(sizeof(int64_t));
    L.off_A = L.off_part + a256(sizeof(double) * (size_t)L.n_mt * n_E);
    L.off_B = L.off_A + a256((size_t)L.n_mt * L.n_kt * nd * TILE_A);
    L.total = L.off_B + a256((size_t)L.n_nt * L.n_kt * nd * TILE_B);
    return L;
}

template <int ND>
cudaError_t run(AmpRef amp, int64_t amp_ld, const double *w, const uint8_t *good, int64_t n_traj,
                int n_steps, double dt, double E_min, double E_max, int n_E, double *I_out,
                int64_t *n_good_out, void *scratch, cudaStream_t s, int *n_launch)
{
    using CF = Cfg<ND>;
    const TcLayout L = tc_layout(ND, n_traj, n_steps, n_E);
    uint8_t *base = static_cast<uint8_t *>(scratch);
    int64_t *ng = reinterpret_cast<int64_t *>(base + L.off_ng);
    double *part = reinterpret_cast<double *>(base + L.off_part);
    uint8_t *At = base + L.off_A;
    uint8_t *Bt = base + L.off_B;
    const double dE = (E_max - E_min) / (n_E - 1);
    const double scale = dt * dt / (kTwoPi * (n_steps * dt));
    cudaError_t e;
    *n_launch = 0;
    k_tc_count_good<<<1, 1024, 0, s>>>(good, n_traj, ng, n_good_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t chunks = (int64_t)L.n_kt * (BK / 8);
    const int64_t na = L.rows_pad * chunks;
    k_split_amp<ND><<<(unsigned)((na + 255) / 256), 256, 0, s>>>(amp, amp_ld, good, n_traj, L.K, L.n_kt,
                                                                 L.rows_pad, At);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t nb = (int64_t)L.n_nt * BN * chunks;
    k_split_tw<ND><<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(L.K, L.n_kt, n_E, L.n_nt, E_min, dE, dt, Bt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_ft_tc<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)L.n_nt, (unsigned)L.n_mt);
    k_ft_tc<ND><<<grid, 128, CF::SMEM, s>>>(At, Bt, w, good, n_traj, L.n_kt, n_E, part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_tc_reduce<<<(n_E + 255) / 256, 256, 0, s>>>(part, (int)L.n_mt, n_E, ng, scale, I_out);
    *n_launch = 5;
    return cudaGetLastError();
}

}  // namespace tc

int ft_tc_digits(int ft_mode)
{
    switch (ft_mode) {
    case SCIVR_FT_TC_BF16: return 1;
    case SCIVR_FT_TC_BF16X3: return 2;
    case SCIVR_FT_TC_BF16X6: return 3;
    default: return 0;
    }
}

size_t spectrum_tc_scratch_bytes(int ft_mode, int64_t n_traj, int n_steps, int n_E)
{
    return tc::tc_layout(ft_tc_digits(ft_mode), n_traj, n_steps, n_E).total;
}

cudaError_t launch_spectrum_tc(int ft_mode, AmpRef amp, int64_t amp_ld, const double *w,
                               const uint8_t *good, int64_t n_traj, int n_steps, double dt, double E_min,
                               double E_max, int n_E, double *I_out, int64_t *n_good_out, void *scratch,
                               cudaStream_t s, int *n_launch)
{
    switch (ft_tc_digits(ft_mode)) {
    case 1: return tc::run<1>(amp, amp_ld, w, good, n_traj, n_steps, dt, E_min, E_max, n_E, I_out, n_good_out, scratch, s, n_launch);
    case 2: return tc::run<2>(amp, amp_ld, w, good, n_traj, n_steps, dt, E_min, E_max, n_E, I_out, n_good_out, scratch, s, n_launch);
    case 3: return tc::run<3>(amp, amp_ld, w, good, n_traj, n_steps, dt, E_min, E_max, n_E, I_out, n_good_out, scratch, s, n_launch);
    default: *n_launch = 0; return cudaErrorInvalidValue;
    }
}

cudaError_t launch_wait_selftest(double seconds, cudaStream_t s)
{
    const long long limit = (long long)(seconds * 2.0e9);   // SM clock cycles at about 2 GHz
    tc::k_wait_selftest<<<1, 32, 0, s>>>(limit);
    return cudaGetLastError();
}

cudaError_t read_and_clear_status(int *status)
{
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(status, g_device_status, sizeof(int));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_device_status, &zero, sizeof(int));
}

}  // namespace scivr
