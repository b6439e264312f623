// Register-resident passes of the cycle (any number of probe modes K; the
// column pass has a one-mode and a K-mode form).
//
// Each line transform N = R * M keeps its data in registers from the global
// load to the global store with a single padded shared-memory transpose:
//
//   thread (line, n1) loads x[n1 + M n2] (n2 < R) straight from global memory,
//   runs an R-point codelet, multiplies by w_N^(n1 k2), writes y[k2 (M+1) + n1];
//   thread (line, k2) reads y[k2 (M+1) + n1] (n1 < M), runs an M-point codelet
//   and holds X[k2 + R k1] (k1 < M) in registers.
//
// The column pass continues in registers: projection and LLK on X, then the
// inverse transform with the roles of R and M swapped (an M-point codelet on
// the values the thread already holds, twiddle, transpose, R-point codelet),
// so that a column makes two shared-memory round trips in total.
#pragma once
#include "kernels.cuh"

namespace ptx {

// Lines per block of the register-resident kernels (rows of a frame for the
// row passes, columns for the column pass).
template <int N>
__host__ __device__ constexpr int reg_lines() {
    return N >= 384 ? 8 : ((N == 192 || N == 80 || N == 160 || N == 224) ? 16 : (4096 / N > N ? N : 4096 / N));
}
// Columns per block of the register column passes: 16 for the large sizes,
// whose 16-point first factor then gives every thread one pass-2 item.
template <int N>
__host__ __device__ constexpr int reg_cols() {
    return (N == 384 || N == 400 || N == 448 || N == 512) ? 16 : reg_lines<N>();
}
// Shared-memory pitch of a line: room for both padded intermediate layouts
// (R (M+1) and M (R+1) elements), odd.
template <int N>
__host__ __device__ constexpr int reg_pitch() {
    return Plan<N>::M == 1 ? N + 1 : N + (Plan<N>::R > Plan<N>::M ? Plan<N>::R : Plan<N>::M) + 1;
}

template <int N>
struct RegShape {
    static constexpr int R = Plan<N>::R, M = Plan<N>::M, L = reg_lines<N>(), P = reg_pitch<N>();
    static constexpr int I1 = (L * M + kThreads - 1) / kThreads;  // pass-1 items per thread
    static constexpr int I2 = (L * R + kThreads - 1) / kThreads;  // pass-2 items per thread
    // the column passes: C columns per block, their items per thread
    static constexpr int C = reg_cols<N>();
    static constexpr int CI1 = (C * M + kThreads - 1) / kThreads;
    static constexpr int CI2 = (C * R + kThreads - 1) / kThreads;
    static_assert(N % C == 0 && CI2 * M <= 32, "columns divide N; a thread's pixels fit the 32 mask bits");
    // blocks per SM the register budget is sized for: large codelets (24, 32
    // points) need more registers per thread
    static constexpr int MinBlocks = (R > M ? R : M) >= 20 ? 2 : 5;
    // the column pass also holds its pixels' intensities in registers
    static constexpr int ColMinBlocks = (R > M ? R : M) >= 20 ? 2 : 4;
    static_assert(M > 1, "register kernels need two passes");
    static_assert(N % L == 0, "lines per block must divide N");
};

// twiddle w_N^(DIR a b), a < R, b < M, from the block's table tw[a * M + b] = w_N^(-a b)
template <int N, int DIR>
__device__ __forceinline__ float2 tw_get(const float2* tw, int a, int b) {
    float2 t = tw[a * Plan<N>::M + b];
    if (DIR > 0) t.y = -t.y;
    return t;
}

// ---------------------------------------------------------------------------
// Row forward: Phi_k = P_k O[r_j], X = Phi_k or 2 Phi_k - Psi_k (kDM), row FFT
// -> spec.  The DM form issues its exit-wave loads (HBM) ahead of the probe
// and object loads (L1 / L2).
// grid (N / L, frames in batch x K); blockIdx.y = frame * K + mode
// ---------------------------------------------------------------------------
template <int N, bool kDM>
__global__ void __launch_bounds__(kThreads, RegShape<N>::MinBlocks) k_row_fwd_r(ProbArgs a, int j0) {
#define PTX_BX blockIdx.x
#define PTX_BY blockIdx.y
#include "body_row_fwd.inc"
#undef PTX_BX
#undef PTX_BY
}

// ---------------------------------------------------------------------------
// Column pass: column FFT, projection + LLK, inverse column FFT.
// grid (N / L, frames in batch); block handles columns [x0, x0 + L).
// ---------------------------------------------------------------------------
// kBg: the problem has an incoherent background (separate instantiation, so
// that the common path carries none of its loads and sums).  kCycle: the
// cycle's projection (COL_PROJECT) fixed at compile time; otherwise the mode
// comes from the argument.
template <int N, bool kBg, bool kCycle>
__global__ void __launch_bounds__(kThreads, RegShape<N>::ColMinBlocks) k_col_r(ProbArgs a, int j0, int mode_arg) {
#define PTX_BX blockIdx.x
#define PTX_BY blockIdx.y
#define PTX_GX gridDim.x
#include "body_col.inc"
#undef PTX_BX
#undef PTX_BY
#undef PTX_GX
}

// ---------------------------------------------------------------------------
// Column pass for K > 1 probe modes.  The projection factor of a pixel is
// common to its modes (sqrt(I_o) / sqrt(sum_k |X^_k|^2)), so the pass runs in
// two sweeps over the modes:
//   1. forward column transform of each mode; the thread sums |X^_k|^2 over
//      the modes for its pixels in registers and writes X^_k back into the
//      stack at those same pixels (L2);
//   2. the factor (and the LLK) per pixel, then for each mode: the thread
//      reloads its own X^_k, scales it, and the inverse column transform
//      writes the mode back.
// The thread-to-pixel mapping is that of k_col_r (so the mask-bit table is
// shared).  grid (N / C, frames in batch).
// ---------------------------------------------------------------------------
// kCycle: the cycle's projection without a background, fixed at compile time.
template <int N, bool kCycle>
__global__ void __launch_bounds__(kThreads, RegShape<N>::ColMinBlocks) k_col_modes_r(ProbArgs a, int j0, int mode_arg) {
    const int mode = kCycle ? (int)COL_PROJECT : mode_arg;
    const float* bgp = kCycle ? nullptr : a.bg;
    using S = RegShape<N>;
    constexpr int R = S::R, M = S::M, C = S::C, P = S::P;
    constexpr int I1b = (C * M + kThreads - 1) / kThreads;  // inverse pass-2 items (M per column)
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red_s[kThreads / 32];
    float2* tw = sm;
    float2* buf = sm + N;
    pdl_launch_dependents();
    load_twiddles<N>(tw);
    const int K = a.K;
    const int x0 = blockIdx.x * C;
    const int b = blockIdx.y;
    const int j = j0 + b;
    float2* spec_b = a.spec + (size_t)b * K * N * N + x0;
    float ic_r[S::CI2][M];  // sum over modes of |X^_k|^2, then the factor
#pragma unroll
    for (int i = 0; i < S::CI2; ++i)
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) ic_r[i][k1] = 0.f;
    __syncthreads();
    // launched as a programmatic dependent of the row pass that writes the work stack
    pdl_wait();
    // sweep 1: forward transforms
    for (int k = 0; k < K; ++k) {
        float2* spec = spec_b + (size_t)k * N * N;
#pragma unroll
        for (int i = 0; i < S::CI1; ++i) {
            const int w = threadIdx.x + i * kThreads;
            if (w < C * M) {
                const int n1 = w / C, c = w - n1 * C;
                float2 v[R];
                const uint64_t el = policy_evict_last();
#pragma unroll
                for (int n2 = 0; n2 < R; ++n2) v[n2] = ld_hint(spec + (size_t)(n1 + M * n2) * N + c, el);
                Dft<R, -1>::run(v);
                float2* o = buf + c * P + n1;
                o[0] = v[0];
#pragma unroll
                for (int k2 = 1; k2 < R; ++k2) o[k2 * (M + 1)] = cmul(v[k2], tw_get<N, -1>(tw, k2, n1));
            }
        }
        __syncthreads();
        float2 u[S::CI2][M];
#pragma unroll
        for (int i = 0; i < S::CI2; ++i) {
            const int w = threadIdx.x + i * kThreads;
            if (w < C * R) {
                const int k2 = w / C, c = w - k2 * C;
                const float2* src = buf + c * P + k2 * (M + 1);
#pragma unroll
                for (int n1 = 0; n1 < M; ++n1) u[i][n1] = src[n1];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < S::CI2; ++i) {
            const int w = threadIdx.x + i * kThreads;
            if (w < C * R) {
                const int k2 = w / C, c = w - k2 * C;
                Dft<M, -1>::run(u[i]);
                const uint64_t el = policy_evict_last();
#pragma unroll
                for (int k1 = 0; k1 < M; ++k1) {
                    ic_r[i][k1] += cnorm(u[i][k1]);
                    st_hint(spec + (size_t)(k2 + R * k1) * N + c, u[i][k1], el);
                }
            }
        }
    }
    // the factor per pixel and the LLK
    constexpr float invN2 = 1.0f / float(N * N);
    float llk = 0.f;  // the terms are >= 0: a plain float sum of a thread's pixels
#pragma unroll
    for (int i = 0; i < S::CI2; ++i) {
        const int w = threadIdx.x + i * kThreads;
        if (w < C * R) {
            const int k2 = w / C, c = w - k2 * C;
            uint32_t mbits = 0u;
            if (a.mbits) mbits = a.mbits[blockIdx.x * kThreads + threadIdx.x] >> (i * M);
            const float* ib = a.iobs + (size_t)j * N * N + (size_t)k2 * N + x0 + c;
#pragma unroll
            for (int k1 = 0; k1 < M; ++k1) {
                const int pix = (k2 + R * k1) * N + x0 + c;
                const bool masked = a.mbits ? ((mbits >> k1) & 1u) != 0u : a.mask[pix] != 0;
                float ic = ic_r[i][k1] * invN2;
                const float io = __ldcs(ib + (size_t)R * k1 * N);
                if (bgp) {
                    ic += __ldg(bgp + pix);
                    if (a.bg_acc && !masked) atomicAdd(a.bg_acc + pix, fmaxf(io, 0.f) / fmaxf(ic, 1e-30f));
                }
                float f;
                if (mode == COL_PROJECT) {
                    float ratio;
                    const float term = llk_term_ratio(ic, io, ratio);
                    if (!masked) llk += term;
                    f = masked ? 0.f : (ratio - 1.0f) * invN2;
                } else {
                    if (!masked) llk += llk_term_fast(ic, io);
                    f = masked ? 0.f : 2.0f * (1.0f - __fdividef(fmaxf(io, 0.f), fmaxf(ic, 1e-30f))) * invN2;
                }
                ic_r[i][k1] = f;
            }
        }
    }
    const double tot = block_sum_pos<kThreads>(llk, red_s);
    if (threadIdx.x == 0) a.llk_part[(size_t)j * gridDim.x + blockIdx.x] = tot;
    if (mode == COL_LLK) return;
    // sweep 2: scale and inverse transforms
    for (int k = 0; k < K; ++k) {
        float2* spec = spec_b + (size_t)k * N * N;
#pragma unroll
        for (int i = 0; i < S::CI2; ++i) {
            const int w = threadIdx.x + i * kThreads;
            if (w < C * R) {
                const int k2 = w / C, c = w - k2 * C;
                float2 u[M];
#pragma unroll
                for (int k1 = 0; k1 < M; ++k1) u[k1] = cscale(spec[(size_t)(k2 + R * k1) * N + c], ic_r[i][k1]);
                // inverse pass 1: M-point codelet over k1, twiddle w_N^(+k2 k2'), y'[k2' (R+1) + k2]
                Dft<M, +1>::run(u);
                float2* o = buf + c * P + k2;
                o[0] = u[0];
#pragma unroll
                for (int kk = 1; kk < M; ++kk) o[kk * (R + 1)] = cmul(u[kk], tw_get<N, +1>(tw, k2, kk));
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < I1b; ++i) {
            const int w = threadIdx.x + i * kThreads;
            if (w < C * M) {
                const int kk = w / C, c = w - kk * C;
                float2 v[R];
                const float2* src = buf + c * P + kk * (R + 1);
#pragma unroll
                for (int n = 0; n < R; ++n) v[n] = src[n];
                Dft<R, +1>::run(v);
                const uint64_t el = policy_evict_last();
#pragma unroll
                for (int k1 = 0; k1 < R; ++k1) st_hint(spec + (size_t)(kk + M * k1) * N + c, v[k1], el);
            }
        }
        __syncthreads();
    }
}

// Factor order of the row-backward transform.  For the large sizes the
// 16-point factor goes second (N = R' M' with M' = 16), so that a thread's
// pass-2 pixels (M' of them) keep the probe, its sums and the object rows in
// registers and shared memory as for the smaller sizes.
template <int N>
struct BwdShape {
    static constexpr bool kSwap = (N == 384 || N == 400 || N == 448 || N == 512);
    static constexpr int R = kSwap ? Plan<N>::M : Plan<N>::R, M = kSwap ? Plan<N>::R : Plan<N>::M;
    static constexpr int L = reg_lines<N>();
    static constexpr int I1 = (L * M + kThreads - 1) / kThreads;
    static constexpr int I2 = (L * R + kThreads - 1) / kThreads;
    static constexpr bool kRegAcc = I2 * M <= 16;  // probe accumulators in registers, else shared memory
    static_assert(R * (M + 1) <= reg_pitch<N>() && M * (R + 1) <= reg_pitch<N>(), "both layouts fit a line");
};
// w_N^(+a b) for a < BwdShape::R, b < BwdShape::M from the table tw[a * M + b] = w_N^(-a b) of Plan<N>
template <int N>
__device__ __forceinline__ float2 tw_bwd(const float2* tw, int a, int b) {
    float2 t = BwdShape<N>::kSwap ? tw[b * Plan<N>::M + a] : tw[a * Plan<N>::M + b];
    t.y = -t.y;
    return t;
}

// ---------------------------------------------------------------------------
// Row backward: inverse row FFT -> D; Psi' = Phi + D stored to the exit-wave
// stack (AP and DM), probe numerator/denominator in registers across the
// block's frames, flushed once.  In gradient mode D is the back-propagated
// weighted wave: G_O is scattered with red.v2, G_P reduced like N_P.
// grid (N / L, G K); blockIdx.y = slot * K + mode: the block handles rows
// [y0, y0 + L) of one probe mode in frames slot + G t.
// ---------------------------------------------------------------------------
// kForm fixes the mode and the flags at compile time: 1 = the cycle's form
// (AP / DM: Psi' stored, probe sums accumulated), 2 = the object gradient
// alone (BWD_GRAD, no probe gradient); 0 = all from the arguments.
template <int N, int kForm>
__global__ void __launch_bounds__(kThreads, 2) k_row_bwd_r(ProbArgs a, int j0, int nb, int mode_arg, int upd_obj_arg,
                                                           int upd_probe_arg) {
#define PTX_BX blockIdx.x
#define PTX_BY blockIdx.y
#define PTX_GY gridDim.y
#include "body_row_bwd.inc"
#undef PTX_BX
#undef PTX_BY
#undef PTX_GY
}

// ---------------------------------------------------------------------------
// ML line search, one probe mode (the same arithmetic as k_row_fwd_ls /
// k_col_ls, with the register-resident transforms).  For a direction (dO, dP)
// the far field along the line is A + a B + a^2 C with A = FT(P O),
// B = FT(dP O + P dO), C = FT(dP dO); C vanishes unless both parts of the
// direction are given.
//
// Row pass: grid (N / L, frames in batch, waves), blockIdx.z = wave (0: A,
// 1: B, 2: C); row transforms into spec[b][wave] (gridDim.z waves per frame).
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kThreads, RegShape<N>::MinBlocks) k_row_fwd_ls_r(ProbArgs a, int j0) {
    using S = RegShape<N>;
    constexpr int R = S::R, M = S::M, L = S::L, P = S::P;
    extern __shared__ __align__(16) float2 sm[];
    float2* tw = sm;
    float2* buf = sm + N;
    pdl_launch_dependents();
    load_twiddles<N>(tw);
    const int y0 = blockIdx.x * L;
    const int b = blockIdx.y;
    const int wave = blockIdx.z;
    const int2 p = a.pos[j0 + b];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < S::I1; ++i) {
        const int w = threadIdx.x + i * kThreads;
        if (w < L * M) {
            const int line = w / M, n1 = w - line * M;
            const int y = y0 + line;
            const size_t pi = (size_t)y * N + n1;
            const size_t oi = (size_t)(p.x + y) * a.Wo + p.y + n1;
            float2 v[R];
#pragma unroll
            for (int n2 = 0; n2 < R; ++n2) {
                const size_t pk = pi + M * n2, ok = oi + M * n2;
                float2 x;
                if (wave == 0) {
                    x = cmul(__ldg(a.probe + pk), __ldg(a.obj + ok));
                } else if (wave == 1) {
                    x = make_float2(0.f, 0.f);
                    if (a.dir_obj) x = cmul(__ldg(a.probe + pk), __ldg(a.dir_obj + ok));
                    if (a.dir_probe) x = cadd(x, cmul(__ldg(a.dir_probe + pk), __ldg(a.obj + ok)));
                } else {
                    x = cmul(__ldg(a.dir_probe + pk), __ldg(a.dir_obj + ok));
                }
                v[n2] = x;
            }
            Dft<R, -1>::run(v);
            float2* o = buf + line * P + n1;
            o[0] = v[0];
#pragma unroll
            for (int k2 = 1; k2 < R; ++k2) o[k2 * (M + 1)] = cmul(v[k2], tw_get<N, -1>(tw, k2, n1));
        }
    }
    __syncthreads();
    // launched as a programmatic dependent of the previous batch's column pass,
    // which reads the work stack: wait before writing it
    pdl_wait();
#pragma unroll
    for (int i = 0; i < S::I2; ++i) {
        const int w = threadIdx.x + i * kThreads;
        if (w < L * R) {
            const int line = w / R, k2 = w - line * R;
            float2 u[M];
            const float2* src = buf + line * P + k2 * (M + 1);
#pragma unroll
            for (int n1 = 0; n1 < M; ++n1) u[n1] = src[n1];
            Dft<M, -1>::run(u);
            float2* dst = a.spec + (((size_t)b * gridDim.z + wave) * N + y0 + line) * N + k2;
            const uint64_t el = policy_evict_last();
#pragma unroll
            for (int k1 = 0; k1 < M; ++k1) st_hint(dst + R * k1, u[k1], el);
        }
    }
}

// Blocks per SM of the line-search column pass: it holds A, the d2I partial
// and one more wave per pixel in registers.
template <int N>
__host__ __device__ constexpr int ls_min_blocks() {
    return Plan<N>::M >= 20 ? 1 : 2;
}

// Column pass: column transforms of the waves (A first, then C, then B, so
// that the reduction runs on B while it is in registers) and the FP64 sums
//   L'(0)  = sum (1 - I_o/I_c) dI,  L''(0) = sum [(1 - I_o/I_c) d2I + (I_o/I_c^2) dI^2]
// with dI = 2 Re(conj(A) B), d2I = 2 |B|^2 + 4 Re(conj(A) C), over unmasked
// pixels; one (L', L'') pair per block into ls_part[j][blockIdx.x].  The
// per-pixel terms are single precision (I_o dI^2 / I_c^2 as I_o (dI / I_c)^2,
// which stays finite at the I_c floor), summed with compensation per thread and
// in FP64 across the block.  grid (N / C, frames in batch).
template <int N>
__global__ void __launch_bounds__(kThreads, ls_min_blocks<N>()) k_col_ls_r(ProbArgs a, int j0, int nwaves) {
    using S = RegShape<N>;
    constexpr int R = S::R, M = S::M, C = S::C, P = S::P;
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red_s[kThreads / 32];
    float2* tw = sm;
    float2* buf = sm + N;
    pdl_launch_dependents();
    load_twiddles<N>(tw);
    const int x0 = blockIdx.x * C;
    const int b = blockIdx.y;
    const int j = j0 + b;
    constexpr float invN2 = 1.0f / float(N * N);
    float2 A[S::CI2][M];
    float d2[S::CI2][M];
    KahanF l1, l2;  // per-pixel terms in single precision (FP64 throughput is low), compensated sums
    __syncthreads();
    // launched as a programmatic dependent of the row pass that writes the work stack
    pdl_wait();
    for (int s = 0; s < nwaves; ++s) {
        const int wave = s == 0 ? 0 : (s == nwaves - 1 ? 1 : 2);
        const float2* spec = a.spec + ((size_t)b * nwaves + wave) * N * N + x0;
#pragma unroll
        for (int i = 0; i < S::CI1; ++i) {
            const int w = threadIdx.x + i * kThreads;
            if (w < C * M) {
                const int n1 = w / C, c = w - n1 * C;
                float2 v[R];
#pragma unroll
                for (int n2 = 0; n2 < R; ++n2) v[n2] = __ldcs(spec + (size_t)(n1 + M * n2) * N + c);
                Dft<R, -1>::run(v);
                float2* o = buf + c * P + n1;
                o[0] = v[0];
#pragma unroll
                for (int k2 = 1; k2 < R; ++k2) o[k2 * (M + 1)] = cmul(v[k2], tw_get<N, -1>(tw, k2, n1));
            }
        }
        __syncthreads();
        float2 u[S::CI2][M];
#pragma unroll
        for (int i = 0; i < S::CI2; ++i) {
            const int w = threadIdx.x + i * kThreads;
            if (w < C * R) {
                const int k2 = w / C, c = w - k2 * C;
                const float2* src = buf + c * P + k2 * (M + 1);
#pragma unroll
                for (int n1 = 0; n1 < M; ++n1) u[i][n1] = src[n1];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < S::CI2; ++i) {
            const int w = threadIdx.x + i * kThreads;
            if (w < C * R) {
                const int k2 = w / C, c = w - k2 * C;
                Dft<M, -1>::run(u[i]);
                if (s == 0) {
#pragma unroll
                    for (int k1 = 0; k1 < M; ++k1) {
                        A[i][k1] = u[i][k1];
                        d2[i][k1] = 0.f;
                    }
                } else if (wave == 2) {
#pragma unroll
                    for (int k1 = 0; k1 < M; ++k1)
                        d2[i][k1] = 4.f * (A[i][k1].x * u[i][k1].x + A[i][k1].y * u[i][k1].y) * invN2;
                } else {
                    uint32_t mbits = 0u;
                    if (a.mbits) mbits = a.mbits[blockIdx.x * kThreads + threadIdx.x] >> (i * M);
                    const float* io_p = a.iobs + (size_t)j * N * N + (size_t)k2 * N + x0 + c;
#pragma unroll
                    for (int k1 = 0; k1 < M; ++k1) {
                        const int pix = (k2 + R * k1) * N + x0 + c;
                        const bool masked = a.mbits ? ((mbits >> k1) & 1u) : (a.mask[pix] != 0);
                        if (masked) continue;
                        const float2 av = A[i][k1], bv = u[i][k1];
                        const float ic = cnorm(av) * invN2 + (a.bg ? __ldg(a.bg + pix) : 0.f);
                        const float di = 2.f * (av.x * bv.x + av.y * bv.y) * invN2;
                        const float dd = d2[i][k1] + 2.f * cnorm(bv) * invN2;
                        const float io = fmaxf(__ldcs(io_p + (size_t)R * k1 * N), 0.f);
                        const float ric = __fdividef(1.0f, fmaxf(ic, 1e-30f));  // 1 / I_c (a few ulp)
                        const float w1 = fmaf(-io, ric, 1.f);
                        const float q = di * ric;  // I_o dI^2 / I_c^2 = I_o q^2
                        l1.add(w1 * di);
                        l2.add(fmaf(w1, dd, io * q * q));
                    }
                }
            }
        }
    }
    const double t1 = block_sum_double<kThreads>(l1.value(), red_s);
    __syncthreads();
    const double t2 = block_sum_double<kThreads>(l2.value(), red_s);
    if (threadIdx.x == 0) {
        double* out = a.ls_part + 2 * ((size_t)j * gridDim.x + blockIdx.x);
        out[0] = t1;
        out[1] = t2;
    }
}

template <int N>
size_t smem_row_fwd_r() { return sizeof(float2) * (N + (size_t)RegShape<N>::L * RegShape<N>::P); }
template <int N>
size_t smem_col_r() {
    using S = RegShape<N>;
    return sizeof(float2) * (N + (size_t)S::C * S::P);
}
template <int N>
size_t smem_row_bwd_r() {
    using S = BwdShape<N>;
    const bool reg_acc = S::kRegAcc;
    return sizeof(float2) * (N + (reg_acc ? 2 : 1) * (size_t)S::L * N + (size_t)S::L * reg_pitch<N>()) +
           (reg_acc ? 0 : (size_t)S::L * N * (sizeof(float2) + sizeof(float)));
}

template <int N>
cudaError_t set_attrs_r() {
    cudaError_t e;
    const int mx = 200 * 1024;
    const int carve = cudaSharedmemCarveoutMaxShared;  // room for 5-6 blocks of ~37 KB per SM
    if ((e = cudaFuncSetAttribute(k_row_fwd_r<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_row_fwd_r<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_col_r<N, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_col_r<N, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_col_r<N, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_col_r<N, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_row_bwd_r<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_row_bwd_r<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_row_bwd_r<N, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_col_modes_r<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_col_modes_r<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_col_modes_r<N, true>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
    if ((e = cudaFuncSetAttribute(k_col_modes_r<N, false>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
    if ((e = cudaFuncSetAttribute(k_row_fwd_ls_r<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_col_ls_r<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_row_fwd_r<N, false>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
    if ((e = cudaFuncSetAttribute(k_row_fwd_r<N, true>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
    if ((e = cudaFuncSetAttribute(k_col_r<N, false, true>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
    if ((e = cudaFuncSetAttribute(k_col_r<N, false, false>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
    if ((e = cudaFuncSetAttribute(k_col_r<N, true, true>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
    if ((e = cudaFuncSetAttribute(k_col_r<N, true, false>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
    if ((e = cudaFuncSetAttribute(k_row_bwd_r<N, 0>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
    if ((e = cudaFuncSetAttribute(k_row_bwd_r<N, 1>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
    if ((e = cudaFuncSetAttribute(k_row_bwd_r<N, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
    return cudaSuccess;
}

}  // namespace ptx
