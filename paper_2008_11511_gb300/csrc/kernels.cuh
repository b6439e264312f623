// Kernels of the far-field ptychography cycle.  One cycle over a batch of
// frames is three passes through a Fourier-space work stack `spec` that is
// sized to stay resident in L2:
//
//   row_fwd   : Phi = P_k . O[r_j] (ObjProbe2Psi), X = Phi (AP) or 2 Phi - Psi (DM),
//               forward FFT of each row                        -> spec
//   col       : forward FFT of each column, then per pixel the amplitude
//               projection (ApplyAmplitude, common factor over modes) and the
//               Poisson LLK, then the inverse column FFT of the correction
//               D^ = P_M(X^) - X^                               -> spec
//   row_bwd   : inverse row FFT -> D = IFT(P_M(FT X)) - X; the new exit wave
//               is Psi' = Phi + D (equal to Psi + P_F(X) - Phi for DM and to
//               P_F(Phi) for AP), scattered into the Psi2ObjProbe numerators
//               and denominators.
//
// After all batches: max of the denominators, normalisation with inertia,
// and the FP64 reduction of the per-block LLK partial sums.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft.cuh"

namespace ptx {

constexpr int kThreads = 256;

enum RowFwdMode : int { X_PHI = 0, X_DM = 1 };
enum ColMode : int { COL_PROJECT = 0, COL_LLK = 1, COL_GRAD = 2 };
enum RowBwdMode : int { BWD_AP = 0, BWD_DM = 1, BWD_GRAD = 2 };

// Device view of one problem (all pointers device, fixed for a handle).
struct ProbArgs {
    int N, K, J, Ho, Wo;
    float2* obj;            // [Ho][Wo]
    float2* probe;          // [K][N][N]
    const float* iobs;      // [J][N][N]
    float2* psi;            // [J][K][N][N] or null
    const int2* pos;        // [J] {row, col}
    const uint8_t* mask;    // [N][N]
    float4* acc_obj;        // [Ho][Wo] {Re N_O, Im N_O, D_O, 0}
    float4* acc_probe;      // [K][N][N] {Re N_P, Im N_P, D_P, 0}
    float2* spec;           // [B][K][N][N] batch work stack
    double* llk_part;       // [J][ncolblk] per-block LLK partial sums
    unsigned* maxbits;      // [2] max D_O, max D_P (float bits; values >= 0)
    float2* grad_obj;       // [Ho][Wo] (ML gradient) or null
    float2* grad_probe;     // [K][N][N] or null
    const float2* dir_obj;  // [Ho][Wo] ML search direction (line-search pass) or null
    const float2* dir_probe;  // [K][N][N] or null
    double* ls_part;        // [J][ncolblk][2] line-search partial sums
    int L1, C2, L3;         // rows per row_fwd block, columns per col block, rows per row_bwd block
    int* err_flag;          // host-mapped flag, set when a bounded device wait gives up (or null)
    const uint32_t* mbits;  // [N / C][256] mask bits per thread of the register column pass
    const float2* nf_t;     // [N] near-field transfer factors t[k] (h[ky][kx] = t[ky] t[kx]) or null
    const float* bg;        // [N][N] incoherent background added to the model intensity, or null
    float* bg_acc;          // [N][N] sum over frames of I_o / (I_c + B) (background update), or null
};

constexpr int kCycleEndBlocks = 64;  // blocks of the cycle's LLK reduction

struct Ctl {
    double* llk_out;  // destination of per-cycle LLK values
    int cycle;        // cycle index within the current call
    int nprob;
    int err;
    unsigned ticket;  // blocks of k_cycle_end done (reset by the last)
    double l2[kCycleEndBlocks];  // k_cycle_end per-block sums
};

// L2 eviction-priority policies (createpolicy) and loads / stores carrying them.
// The Fourier work stack of a batch is written and re-read by the three passes
// and must stay in L2; everything touched once (exit waves read or written,
// intensities, the stack's last read) is marked evict-first so it does not push
// the stack out.
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialisation attribute may start while the previous kernel of its
// stream runs; it signals its own dependents early (launch_dependents) and
// waits for the previous kernel's completion and memory (wait) before its
// first access to what that kernel writes or reads.  Both are no-ops in a
// kernel launched without the attribute.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ float2 ld_hint(const float2* ptr, uint64_t pol) {
    float2 v;
    asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint(float2* ptr, float2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(ptr), "f"(v.x), "f"(v.y), "l"(pol)
                 : "memory");
}
// 16-byte cp.async with an L2 policy
__device__ __forceinline__ void cp_async16_hint(void* smem_dst, const void* gmem_src, uint64_t pol) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem_src), "l"(pol)
                 : "memory");
}

// Asynchronous 8-byte global -> shared copy (cp.async).
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void red_add_v4(float4* addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}
__device__ __forceinline__ void red_add_v2(float2* addr, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b) : "memory");
}

// Poisson LLK of one pixel (deviance form): I_c - I_o + I_o ln(I_o / I_c), = I_c for I_o <= 0,
// I_c floored at 1e-30.  With u = I_c / I_o - 1 the term is I_o (u - ln(1 + u)); for
// -1/2 < u < 1 it is evaluated without cancellation from ln(1+u) = 2 atanh(t),
// t = u / (2 + u):  u - ln(1 + u) = u t - 2 t^3 (1/3 + t^2/5 + t^4/7 + ...), |t| <= 1/3.
__device__ __forceinline__ float llk_term(float ic, float io) {
    if (!(io > 0.f)) return ic;
    float icf = fmaxf(ic, 1e-30f);
    float u = (icf - io) / io;
    float f;
    if (u > -0.5f && u < 1.0f) {
        float t = u / (2.0f + u);
        float t2 = t * t;
        float poly = fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, 1.f / 15.f, 1.f / 13.f), 1.f / 11.f),
                                                     1.f / 9.f), 1.f / 7.f), 1.f / 5.f), 1.f / 3.f);
        f = fmaf(u, t, -2.0f * t * t2 * poly);
    } else {
        f = u - logf(icf / io);
    }
    return io * f;
}

// The same term with hardware-approximate division and logarithm (each a few
// ulp): u, t by __fdividef, ln by __logf in the branch where |u - ln(1+u)| is
// at least 0.19 |u|, so the term keeps a relative error of a few 1e-7.
__device__ __forceinline__ float llk_term_fast(float ic, float io) {
    // both forms are evaluated and the right one selected: no branches (a warp
    // usually holds pixels of both kinds); for io <= 0 the selects discard the
    // non-finite intermediates
    const float icf = fmaxf(ic, 1e-30f);
    const float rio = __fdividef(1.0f, io);
    const float u = (icf - io) * rio;
    const float t = __fdividef(u, 2.0f + u);
    const float t2 = t * t;
    const float poly = fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, 1.f / 15.f, 1.f / 13.f), 1.f / 11.f),
                                                       1.f / 9.f), 1.f / 7.f), 1.f / 5.f), 1.f / 3.f);
    const float fs = fmaf(u, t, -2.0f * t * t2 * poly);
    const float fl = u - __logf(icf * rio);
    const float f = (u > -0.5f && u < 1.0f) ? fs : fl;
    return io > 0.f ? io * f : ic;
}

// The LLK term of llk_term_fast and, from the same quotient, the amplitude
// factor sqrt(max(io, 0) / max(ic, 1e-30)) of the projection: with
// q = max(ic, 1e-30) / io (= 1 + u), the factor is rsqrt(q), one reciprocal
// square root (0 where io <= 0).  Where the oracle's floor differs
// (ic < 1e-30) the model wave is below 1e-15 in modulus and the projected
// value rounds to the same result.
__device__ __forceinline__ float llk_term_ratio(float ic, float io, float& ratio) {
    const float icf = fmaxf(ic, 1e-30f);
    const float rio = __fdividef(1.0f, io);
    const float u = (icf - io) * rio;
    const float t = __fdividef(u, 2.0f + u);
    const float t2 = t * t;
    const float poly = fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, 1.f / 15.f, 1.f / 13.f), 1.f / 11.f),
                                                       1.f / 9.f), 1.f / 7.f), 1.f / 5.f), 1.f / 3.f);
    const float fs = fmaf(u, t, -2.0f * t * t2 * poly);
    const float q = icf * rio;
    const float fl = u - __logf(q);
    const float f = (u > -0.5f && u < 1.0f) ? fs : fl;
    ratio = io > 0.f ? rsqrtf(q) : 0.f;
    return io > 0.f ? io * f : ic;
}

// sqrt(max(io, 0)) / max(sqrt(ic), 1e-20): the amplitude-projection factor, with
// reciprocal square roots (<= 2 ulp each); ic below 1e-40 keeps the floor.
__device__ __forceinline__ float amp_ratio(float io, float ic) {
    const float iop = fmaxf(io, 0.f);
    const float sq_io = iop > 0.f ? iop * rsqrtf(iop) : 0.f;
    return ic > 1e-38f ? sq_io * rsqrtf(ic) : sq_io * 1e20f;
}

// Kahan-compensated float accumulation (per thread), reduced in FP64 across the block.
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        float y = v - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <int T>
__device__ __forceinline__ double block_sum_double(double v, double* red_smem) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red_smem[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (threadIdx.x < T / 32) ? red_smem[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;  // valid in thread 0
}

// Block sum of per-thread partial sums that are >= 0 (LLK terms): a tree of
// warp shuffles in FP32 (five levels, relative error <= 5 u on top of the
// threads' own sums), then the warps' sums in FP64 by thread 0.  Leaves the
// FP64 pipe almost idle (one conversion per warp, T / 32 additions).
template <int T>
__device__ __forceinline__ double block_sum_pos(float v, double* red_smem) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red_smem[warp] = (double)v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < T / 32; ++w) r += red_smem[w];
    }
    return r;  // valid in thread 0
}

// Inter-pass twiddles of the line FFT, tw_s[k2 * M + n1] = exp(-2 pi i n1 k2 / N),
// computed per block with sincospif on the exactly reduced integer n1 k2 mod N.
template <int N>
__device__ __forceinline__ void load_twiddles(float2* tw_s) {
    constexpr int M = Plan<N>::M;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int k2 = i / M, n1 = i - k2 * M;
        const int m = (n1 * k2) % N;
        float s, c;
        sincospif(-2.0f * (float)m / (float)N, &s, &c);
        tw_s[i] = make_float2(c, s);
    }
}

// Max lines (of N elements) held by one block.
template <int N>
__host__ __device__ constexpr int max_lines() {
    return (4096 / N) < 1 ? 1 : ((4096 / N) > 256 ? 256 : (4096 / N));
}

// ---------------------------------------------------------------------------
// row_fwd: grid (N / L1, frames in batch); block handles rows [y0, y0 + L1) of
// all K modes of frame j0 + blockIdx.y.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kThreads) k_row_fwd(ProbArgs a, int j0, int mode) {
    constexpr int P = line_pitch<N>();
    extern __shared__ __align__(16) float2 sm[];
    float2* tw = sm;
    float2* buf = sm + N;
    const int K = a.K, L = a.L1;
    const int y0 = blockIdx.x * L;
    const int b = blockIdx.y;
    const int j = j0 + b;
    load_twiddles<N>(tw);
    const int2 p = a.pos[j];
    const int nel = K * L * N;
    for (int e = threadIdx.x; e < nel; e += kThreads) {
        const int x = e % N;
        const int line = e / N;
        const int k = line / L, r = line - k * L;
        const int y = y0 + r;
        float2 pr = a.probe[((size_t)k * N + y) * N + x];
        float2 ob = a.obj[(size_t)(p.x + y) * a.Wo + (p.y + x)];
        float2 X = cmul(pr, ob);
        if (mode == X_DM) {
            float2 ps = a.psi[(((size_t)j * K + k) * N + y) * N + x];
            X = make_float2(2.f * X.x - ps.x, 2.f * X.y - ps.y);
        }
        buf[line * P + x] = X;
    }
    __syncthreads();
    fft_lines<N, -1, kThreads, max_lines<N>()>(buf, K * L, tw);
    for (int e = threadIdx.x; e < nel; e += kThreads) {
        const int x = e % N;
        const int line = e / N;
        const int k = line / L, r = line - k * L;
        a.spec[(((size_t)b * K + k) * N + y0 + r) * N + x] = buf[line * P + x];
    }
}

// ---------------------------------------------------------------------------
// col: grid (N / C2, frames in batch); block handles columns [x0, x0 + C2) of
// all K modes of one frame.  Lines in shared memory are columns.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kThreads) k_col(ProbArgs a, int j0, int mode) {
    constexpr int P = line_pitch<N>();
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red_s[kThreads / 32];
    float2* tw = sm;
    float2* buf = sm + N;
    const int K = a.K, C = a.C2;
    const int x0 = blockIdx.x * C;
    const int b = blockIdx.y;
    const int j = j0 + b;
    load_twiddles<N>(tw);
    const int nel = K * N * C;
    for (int e = threadIdx.x; e < nel; e += kThreads) {
        const int c = e % C;
        const int t = e / C;
        const int n = t % N, k = t / N;
        buf[(k * C + c) * P + n] = a.spec[(((size_t)b * K + k) * N + n) * N + x0 + c];
    }
    __syncthreads();
    fft_lines<N, -1, kThreads, max_lines<N>()>(buf, K * C, tw);
    constexpr float invN2 = 1.0f / float(N * N);
    KahanF llk;
    const float* io_row = a.iobs + (size_t)j * N * N;
    for (int e = threadIdx.x; e < N * C; e += kThreads) {
        const int c = e % C, n = e / C;
        float icr = 0.f;
        for (int k = 0; k < K; ++k) icr += cnorm(buf[(k * C + c) * P + n]);
        const float ic = icr * invN2 + (a.bg ? a.bg[n * N + x0 + c] : 0.f);
        const float io = io_row[n * N + x0 + c];
        const bool masked = a.mask[n * N + x0 + c] != 0;
        if (!masked) llk.add(llk_term(ic, io));
        if (a.bg_acc && !masked) atomicAdd(a.bg_acc + n * N + x0 + c, fmaxf(io, 0.f) / fmaxf(ic, 1e-30f));
        if (mode != COL_LLK) {
            float f;
            if (masked) {
                f = 0.f;
            } else if (mode == COL_PROJECT) {
                f = (sqrtf(fmaxf(io, 0.f)) / fmaxf(sqrtf(ic), 1e-20f) - 1.0f) * invN2;
            } else {
                f = 2.0f * (1.0f - fmaxf(io, 0.f) / fmaxf(ic, 1e-30f)) * invN2;
            }
            for (int k = 0; k < K; ++k) {
                float2& v = buf[(k * C + c) * P + n];
                v = cscale(v, f);
            }
        }
    }
    double tot = block_sum_double<kThreads>(llk.value(), red_s);
    if (threadIdx.x == 0) a.llk_part[(size_t)j * gridDim.x + blockIdx.x] = tot;
    if (mode == COL_LLK) return;
    __syncthreads();
    fft_lines<N, +1, kThreads, max_lines<N>()>(buf, K * C, tw);
    for (int e = threadIdx.x; e < nel; e += kThreads) {
        const int c = e % C;
        const int t = e / C;
        const int n = t % N, k = t / N;
        a.spec[(((size_t)b * K + k) * N + n) * N + x0 + c] = buf[(k * C + c) * P + n];
    }
}

// ---------------------------------------------------------------------------
// row_bwd: grid (N / L3, G); block handles rows [y0, y0 + L3) of frames
// b = blockIdx.y, blockIdx.y + G, ... of the batch: inverse row FFT, Psi' =
// Phi + D stored, its share of the probe numerator / denominator kept in
// shared memory across those frames (gradient mode: G_O scattered, G_P reduced).
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kThreads) k_row_bwd(ProbArgs a, int j0, int nb, int mode, int upd_obj,
                                                      int upd_probe) {
    constexpr int P = line_pitch<N>();
    extern __shared__ __align__(16) float2 sm[];
    const int K = a.K, L = a.L3;
    float2* tw = sm;
    float2* buf = sm + N;
    float2* np_s = buf + K * L * P;        // [K][L][N]
    float* dp_s = (float*)(np_s + K * L * N);  // [L][N]
    const int y0 = blockIdx.x * L;
    load_twiddles<N>(tw);
    const bool acc_p = upd_probe != 0;
    const bool acc_o = upd_obj != 0;
    if (acc_p) {
        for (int e = threadIdx.x; e < K * L * N; e += kThreads) np_s[e] = make_float2(0.f, 0.f);
        for (int e = threadIdx.x; e < L * N; e += kThreads) dp_s[e] = 0.f;
    }
    const int nel = K * L * N;
    for (int b = blockIdx.y; b < nb; b += gridDim.y) {
        const int j = j0 + b;
        const int2 p = a.pos[j];
        for (int e = threadIdx.x; e < nel; e += kThreads) {
            const int x = e % N;
            const int line = e / N;
            const int k = line / L, r = line - k * L;
            buf[line * P + x] = a.spec[(((size_t)b * K + k) * N + y0 + r) * N + x];
        }
        __syncthreads();
        fft_lines<N, +1, kThreads, max_lines<N>()>(buf, K * L, tw);
        for (int e = threadIdx.x; e < L * N; e += kThreads) {
            const int x = e % N, r = e / N;
            const int y = y0 + r;
            const size_t oidx = (size_t)(p.x + y) * a.Wo + (p.y + x);
            const float2 ob = a.obj[oidx];
            float2 no = make_float2(0.f, 0.f);
            for (int k = 0; k < K; ++k) {
                const float2 d = buf[(k * L + r) * P + x];
                const float2 pr = a.probe[((size_t)k * N + y) * N + x];
                float2 w;
                if (mode == BWD_GRAD) {
                    w = d;
                    if (acc_o) {
                        const float2 t = cconjmul(pr, w);
                        no.x += t.x;
                        no.y += t.y;
                    }
                } else {
                    w = cadd(cmul(pr, ob), d);
                    a.psi[(((size_t)j * K + k) * N + y) * N + x] = w;
                }
                if (acc_p) {
                    const float2 t = cconjmul(ob, w);
                    float2& q = np_s[(k * L + r) * N + x];
                    q.x += t.x;
                    q.y += t.y;
                }
            }
            if (acc_p) dp_s[r * N + x] += cnorm(ob);
            if (acc_o && mode == BWD_GRAD) red_add_v2(a.grad_obj + oidx, no.x, no.y);
        }
        __syncthreads();
    }
    if (acc_p) {
        for (int e = threadIdx.x; e < K * L * N; e += kThreads) {
            const int x = e % N;
            const int line = e / N;
            const int k = line / L, r = line - k * L;
            const size_t pidx = ((size_t)k * N + y0 + r) * N + x;
            const float2 q = np_s[e];
            if (mode == BWD_GRAD)
                red_add_v2(a.grad_probe + pidx, q.x, q.y);
            else
                red_add_v4(a.acc_probe + pidx, q.x, q.y, dp_s[r * N + x], 0.f);
        }
    }
}

// ---------------------------------------------------------------------------
// ML line search.  For a search direction (dO, dP) the far field along the line
// is FT((P + a dP)(O + a dO)) = A + a B + a^2 C with A = FT(P O),
// B = FT(dP O + P dO), C = FT(dP dO).  k_row_fwd_ls writes the row transforms of
// the three waves of every mode (3K lines per frame row: A modes, B modes, C
// modes) and k_col_ls finishes the column transforms and reduces
//   L'(0)  = sum (1 - I_o/I_c) dI,  L''(0) = sum [(1 - I_o/I_c) d2I + (I_o/I_c^2) dI^2]
// with dI = 2 sum_k Re(conj(A) B), d2I = 2 sum_k (|B|^2 + 2 Re(conj(A) C)), in FP64.
// grid (N / L, frames in batch); L rows (columns) of 3K lines per block.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kThreads) k_row_fwd_ls(ProbArgs a, int j0, int L) {
    constexpr int P = line_pitch<N>();
    extern __shared__ __align__(16) float2 sm[];
    float2* tw = sm;
    float2* buf = sm + N;
    const int K = a.K, K3 = 3 * a.K;
    const int y0 = blockIdx.x * L;
    const int b = blockIdx.y;
    const int2 p = a.pos[j0 + b];
    load_twiddles<N>(tw);
    const int nel = 3 * L * N;  // one mode at a time: lines (part, row)
    for (int k = 0; k < K; ++k) {
        for (int e = threadIdx.x; e < nel; e += kThreads) {
            const int x = e % N;
            const int line = e / N;
            const int part = line / L, r = line - part * L;
            const int y = y0 + r;
            const size_t pidx = ((size_t)k * N + y) * N + x;
            const size_t oidx = (size_t)(p.x + y) * a.Wo + (p.y + x);
            const float2 pr = a.probe[pidx], ob = a.obj[oidx];
            const float2 dp = a.dir_probe ? a.dir_probe[pidx] : make_float2(0.f, 0.f);
            const float2 dob = a.dir_obj ? a.dir_obj[oidx] : make_float2(0.f, 0.f);
            float2 v;
            if (part == 0)
                v = cmul(pr, ob);
            else if (part == 1)
                v = cadd(cmul(dp, ob), cmul(pr, dob));
            else
                v = cmul(dp, dob);
            buf[line * P + x] = v;
        }
        __syncthreads();
        fft_lines<N, -1, kThreads, max_lines<N>()>(buf, 3 * L, tw);
        for (int e = threadIdx.x; e < nel; e += kThreads) {
            const int x = e % N;
            const int line = e / N;
            const int part = line / L, r = line - part * L;
            a.spec[(((size_t)b * K3 + part * K + k) * N + y0 + r) * N + x] = buf[line * P + x];
        }
        __syncthreads();
    }
}

template <int N>
__global__ void __launch_bounds__(kThreads) k_col_ls(ProbArgs a, int j0, int C) {
    constexpr int P = line_pitch<N>();
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red_s[kThreads / 32];
    float2* tw = sm;
    float2* buf = sm + N;                        // [3][C] lines of one mode
    float* acc = (float*)(buf + 3 * C * P);      // [3][N * C]: I_c, dI, d2I summed over modes
    const int K = a.K, K3 = 3 * a.K;
    const int x0 = blockIdx.x * C;
    const int b = blockIdx.y;
    const int j = j0 + b;
    load_twiddles<N>(tw);
    for (int e = threadIdx.x; e < 3 * N * C; e += kThreads) acc[e] = 0.f;
    const int nel = 3 * N * C;
    for (int k = 0; k < K; ++k) {
        for (int e = threadIdx.x; e < nel; e += kThreads) {
            const int c = e % C;
            const int t = e / C;
            const int n = t % N, part = t / N;
            buf[(part * C + c) * P + n] = a.spec[(((size_t)b * K3 + part * K + k) * N + n) * N + x0 + c];
        }
        __syncthreads();
        fft_lines<N, -1, kThreads, max_lines<N>()>(buf, 3 * C, tw);
        for (int e = threadIdx.x; e < N * C; e += kThreads) {
            const int c = e % C, n = e / C;
            const float2 A = buf[c * P + n];
            const float2 B = buf[(C + c) * P + n];
            const float2 Cc = buf[(2 * C + c) * P + n];
            acc[e] += cnorm(A);
            acc[N * C + e] += 2.f * (A.x * B.x + A.y * B.y);
            acc[2 * N * C + e] += 2.f * (cnorm(B) + 2.f * (A.x * Cc.x + A.y * Cc.y));
        }
        __syncthreads();
    }
    constexpr float invN2 = 1.0f / float(N * N);
    KahanF l1, l2;  // single-precision terms, compensated sums (as k_col_ls_r)
    const float* io_row = a.iobs + (size_t)j * N * N;
    for (int e = threadIdx.x; e < N * C; e += kThreads) {
        const int c = e % C, n = e / C;
        if (a.mask[n * N + x0 + c]) continue;
        const float ic = acc[e] * invN2 + (a.bg ? a.bg[n * N + x0 + c] : 0.f);
        const float di = acc[N * C + e] * invN2, d2i = acc[2 * N * C + e] * invN2;
        const float io = fmaxf(io_row[n * N + x0 + c], 0.f);
        const float icf = fmaxf(ic, 1e-30f);
        const float w1 = 1.f - io / icf;
        const float q = di / icf;
        l1.add(w1 * di);
        l2.add(fmaf(w1, d2i, io * q * q));
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

// ---------------------------------------------------------------------------
// Normalisation (Psi2ObjProbe second half) and reductions.
// ---------------------------------------------------------------------------
// Object tiles of the gather: kObjTileW x th pixels, one block each, th =
// kObjTileH, or a half or a quarter of it for objects with few tiles (more
// blocks).  Wide tiles make every frame's share of a tile a few long row
// segments (kObjTileW * 8 bytes each), which HBM serves more efficiently than
// short ones.
#ifndef PTX_OBJ_TILE_W
#define PTX_OBJ_TILE_W 32
#endif
constexpr int kObjTileW = PTX_OBJ_TILE_W;
constexpr int kObjTileH = 1024 / kObjTileW;
static_assert(kObjTileW % 32 == 0 && kObjTileW <= 256 && kObjTileH * kObjTileW == 1024, "1024-pixel tiles, 32-wide multiples");
struct TileLists {
    const int* tile_ids;     // [ntiles] tile index ty * ntx + tx of each active tile
    const int* tile_ptr;     // [ntiles + 1] CSR offsets into tile_frames
    const int* tile_frames;  // frames j whose patch meets the tile, ascending
    int ntx;                 // tiles per object row
    int th;                  // tile height (kObjTileH, kObjTileH / 2 or kObjTileH / 4)
};
__global__ void k_obj_gather(ProbArgs a, TileLists tl, int fuse_max);
// Column pass with the 16-point DFT stages on the tensor cores (tcgen05, TF32
// hi + lo split; N = 256, one mode), the split-precision form of k_col_r<256>.
// Persistent schedule of the cycle's batch passes (persistent.cu).  A segment
// is the run of work items of one pass of one batch; items are numbered in
// list order and a segment's start is the number of its first item.
constexpr int kPersSlots = 3;  // work-stack slots (batches in flight)
constexpr int kPersFrames = 4;  // frames per forward-row and column item
struct PSeg {
    int g;       // batch
    int pass;    // 0 forward row pass, 1 column pass, 2 backward row pass
    int start;   // first item
    int pad;
};
struct PBatch {
    int prob;      // problem index
    int j0, nb;    // first frame and frame count
    int G;         // frame slots of the backward row pass
    unsigned n[3]; // items of each pass
    int pad;
};
struct PCtl {
    unsigned head;  // next item to hand out
    int abort;      // set by a wait that gave up: blocks stop taking items
};
struct PersArgs {
    const PSeg* seg;
    int nseg, nitems;
    const PBatch* batch;
    int nbatch;
    const ProbArgs* prob;   // [problems] (spec set per batch from its slot)
    float2* spec;           // slot 0 of the work stack
    size_t slot_elems;      // complex elements per slot
    PCtl* ctl;              // zeroed before each launch
    unsigned* done;         // [3 nbatch] finished items per (batch, pass), zeroed before each launch
    int* err_flag;          // host-mapped error flag or null
    unsigned long long dm_mask;  // problems whose forward pass forms 2 Phi - Psi
    int init;               // DM's first cycle (Psi = Phi): forward passes form Phi
};
size_t pers_smem();
bool pers_supported_N(int N);
cudaError_t set_attrs_persistent();
int pers_blocks_per_sm();
void launch_cycle_persistent(const PersArgs& pa, int grid, cudaStream_t s);

// Number formats of the tensor-core column pass (ptx_set_param "tc" and the
// PTX_FORM_* cycle flags): TF32 hi + lo, BF16 hi + mid + lo, BF16 hi + lo.
enum TcForm : int { TC_NONE = 0, TC_TF32X2 = 1, TC_BF16X3 = 2, TC_BF16X2 = 3 };
// selftest != 0 (256^2 forms): one stage of the first frame issues no MMAs, so
// its bounded wait runs out and the launch reports through err_flag.
void launch_col_tc(const ProbArgs& a, int j0, int nb, int form, int selftest, cudaStream_t s);
cudaError_t set_attrs_tc();
// The row passes with their DFT stages on the tensor cores (256^2, one mode):
// the same work-stack layout as k_row_fwd_r<256> / k_row_bwd_r<256, 1>.
void launch_row_fwd_tc(const ProbArgs& a, int j0, int nb, bool dm, int form, cudaStream_t s);
void launch_row_bwd_tc(const ProbArgs& a, int j0, int nb, int G, int upd_probe, int form, cudaStream_t s);
cudaError_t set_attrs_row_tc();
// SMs of the current device (api.cu)
int sm_count();
// The same gather fed by 3D tensor copies (32 x 32 tiles, N >= 64).
void launch_obj_gather_tma(const void* tm_psi, const void* tm_probe, const ProbArgs& a, const TileLists& tl,
                           int ntiles, int fuse_max, cudaStream_t s);
cudaError_t set_attrs_gather_tma();
__global__ void k_den_max(ProbArgs a, int upd_obj, int upd_probe);
__global__ void k_bg_update(float* bg, float* acc, const uint8_t* mask, int n, float inv_j);
// position refinement (position.cu)
__global__ void k_pos_sums(ProbArgs a, double* part);
__global__ void k_pos_solve(const double* part, int J, int bands, float filter_ratio, float* shifts);
__global__ void k_normalise(ProbArgs a, float alpha_obj, float alpha_probe, int upd_obj, int upd_probe);
__global__ void k_llk_reduce(ProbArgs a, int nparts_per_frame, double* out);
__global__ void k_cycle_end(Ctl* ctl, ProbArgs a, int p, int nparts_per_frame, int last_problem);
__global__ void k_set_ctl(Ctl* ctl, double* llk_out, int nprob);

// ML conjugate-gradient vector steps.  cg[0..2] receive <G,G>, <G,Gp>, <Gp,Gp>
// (Re sum conj(a) b over object and probe), cg[3..4] the line-search L'(0), L''(0).
constexpr int kCgBlocks = 4 * 152;  // blocks of the CG vector kernels

struct CgArgs {
    float2* g_obj;
    float2* g_probe;
    float2* gp_obj;   // previous gradient
    float2* gp_probe;
    float2* d_obj;    // search direction
    float2* d_probe;
    size_t n_obj, n_probe;
    double* cg;       // [8] device scalars
    double* cg_part;  // [kCgBlocks][3] per-block partial dot products
};
__global__ void k_wait_selftest(int* err_flag, unsigned long long limit_ns);
__global__ void k_counts_to_float(const uint16_t* __restrict__ src, float* __restrict__ dst, size_t n);
__global__ void k_counts8_to_float(const uint8_t* __restrict__ src, float* __restrict__ dst, size_t n);
__global__ void k_counts8_escapes(const uint32_t* __restrict__ index, const uint16_t* __restrict__ value,
                                  float* __restrict__ dst, size_t n_esc, size_t n);
__global__ void k_fma_peak(float* __restrict__ sink, int iters, float a, float b);
__global__ void k_cg_dots(CgArgs c);
__global__ void k_cg_reduce(CgArgs c);
__global__ void k_cg_direction(CgArgs c);
__global__ void k_cg_step(CgArgs c, float2* obj, float2* probe);
__global__ void k_ls_reduce(const double* part, size_t nparts, double* out);

// ---------------------------------------------------------------------------
// Plain orthonormal 2D FFT of frames in place (FT / IFT operators).
// ---------------------------------------------------------------------------
template <int N, int DIR>
__global__ void __launch_bounds__(kThreads) k_fft_rows(float2* data, int L) {
    constexpr int P = line_pitch<N>();
    extern __shared__ __align__(16) float2 sm[];
    float2* tw = sm;
    float2* buf = sm + N;
    load_twiddles<N>(tw);
    float2* base = data + ((size_t)blockIdx.y * N + blockIdx.x * L) * N;
    for (int e = threadIdx.x; e < L * N; e += kThreads) buf[(e / N) * P + (e % N)] = base[e];
    __syncthreads();
    fft_lines<N, DIR, kThreads, max_lines<N>()>(buf, L, tw);
    for (int e = threadIdx.x; e < L * N; e += kThreads) base[e] = buf[(e / N) * P + (e % N)];
}

template <int N, int DIR>
__global__ void __launch_bounds__(kThreads) k_fft_cols(float2* data, int C) {
    constexpr int P = line_pitch<N>();
    extern __shared__ __align__(16) float2 sm[];
    float2* tw = sm;
    float2* buf = sm + N;
    load_twiddles<N>(tw);
    float2* base = data + (size_t)blockIdx.y * N * N + blockIdx.x * C;
    for (int e = threadIdx.x; e < N * C; e += kThreads) {
        const int c = e % C, n = e / C;
        buf[c * P + n] = base[(size_t)n * N + c];
    }
    __syncthreads();
    fft_lines<N, DIR, kThreads, max_lines<N>()>(buf, C, tw);
    constexpr float invN = 1.0f / float(N);
    for (int e = threadIdx.x; e < N * C; e += kThreads) {
        const int c = e % C, n = e / C;
        base[(size_t)n * N + c] = cscale(buf[c * P + n], invN);
    }
}

// Launch table for one frame size.  The row_fwd / col / row_bwd entries pick
// the register-resident kernels (kernels_reg.cuh) for the two-pass sizes (any
// number of probe modes), and the shared-memory kernels above for the one-pass
// sizes 8, 12 and 16.
struct KernelSet {
    int N;
    // pdl: launch as a programmatic dependent of the previous kernel of the
    // stream (register kernels only, whose bodies wait for it before touching
    // the work stack); the caller sets it only where that kernel is a batch pass
    void (*row_fwd)(const ProbArgs&, int j0, int nb, int mode, cudaStream_t, bool pdl);
    void (*col)(const ProbArgs&, int j0, int nb, int mode, cudaStream_t, bool pdl);
    void (*row_bwd)(const ProbArgs&, int j0, int nb, int G, int mode, int upd_obj, int upd_probe, cudaStream_t,
                    bool pdl);
    void (*fft2)(float2* data, int nframes, int dir, cudaStream_t);
    // line search; pdl as for the passes above (one-mode register kernels)
    void (*row_fwd_ls)(const ProbArgs&, int j0, int nb, int pdl, cudaStream_t);
    void (*col_ls)(const ProbArgs&, int j0, int nb, int pdl, cudaStream_t);
    int max_lines;  // lines per block of the shared-memory kernels
    int ls_lines;   // rows / columns per block of the line-search kernels
    int reg_lines;  // lines per block of the register kernels (0: none for this N)
    int reg_cols;   // columns per block of the register column passes
    int (*row_bwd_per_sm)();  // resident row-backward blocks per SM (0: not known yet)
    int R, M;
    // column pass fed by tensor copies (K = 1; null where N has none) and its persistent grid
    void (*col_tma)(const void* tm_spec, const void* tm_io, const void* tm_mask, const ProbArgs&, int j0, int nb,
                    int grid, cudaStream_t);
    int (*col_tma_grid)();
    // near-field passes (K = 1, N with two-pass transforms)
    void (*col_nf)(const ProbArgs&, int nb, int dir, cudaStream_t);
    void (*row_proj)(const ProbArgs&, int j0, int nb, int llk_only, cudaStream_t);
};

const KernelSet* kernel_set(int N);
// Whether the register-resident kernels serve a problem with K modes (they
// exist for every two-pass size N, any K).
inline bool use_reg_kernels(const KernelSet* ks, int K) { return K >= 1 && ks->reg_lines > 0; }
// Columns per block of the line-search column pass (register form for one mode).
inline int ls_cols(const KernelSet* ks, int K) { return (K == 1 && ks->reg_lines > 0) ? ks->reg_cols : ks->ls_lines; }

template <int N>
size_t smem_row_fwd_t(int K, int L) { return sizeof(float2) * (N + (size_t)K * L * line_pitch<N>()); }
template <int N>
size_t smem_col_t(int K, int C) { return sizeof(float2) * (N + (size_t)K * C * line_pitch<N>()); }
template <int N>
size_t smem_row_bwd_t(int K, int L) {
    return sizeof(float2) * (N + (size_t)K * L * line_pitch<N>() + (size_t)K * L * N) + sizeof(float) * (size_t)L * N;
}

}  // namespace ptx
#include "kernels_reg.cuh"
#include "kernels_tma.cuh"
#include "kernels_nf.cuh"
namespace ptx {

template <int N>
constexpr bool has_reg() { return Plan<N>::M > 1; }


// Launch k with kThreads threads, as a programmatic dependent of the previous
// kernel of the stream when pdl is set.
template <typename... KArgs, typename... Args>
void launch_dep(void (*k)(KArgs...), dim3 grid, size_t smem, cudaStream_t s, bool pdl, Args... args) {
    if (!pdl) {
        k<<<grid, kThreads, smem, s>>>(args...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, args...);
}

template <int N>
void launch_row_fwd(const ProbArgs& a, int j0, int nb, int mode, cudaStream_t s, bool pdl) {
    if constexpr (has_reg<N>()) {
        dim3 grid(N / RegShape<N>::L, nb * a.K);
        if (mode == X_DM)
            launch_dep(k_row_fwd_r<N, true>, grid, smem_row_fwd_r<N>(), s, pdl, a, j0);
        else
            launch_dep(k_row_fwd_r<N, false>, grid, smem_row_fwd_r<N>(), s, pdl, a, j0);
        return;
    }
    dim3 grid(N / a.L1, nb);
    k_row_fwd<N><<<grid, kThreads, smem_row_fwd_t<N>(a.K, a.L1), s>>>(a, j0, mode);
}
template <int N>
void launch_col(const ProbArgs& a, int j0, int nb, int mode, cudaStream_t s, bool pdl) {
    if constexpr (has_reg<N>()) {
        dim3 grid(N / RegShape<N>::C, nb);
        if (a.K > 1) {
            if (mode == COL_PROJECT && !a.bg)
                launch_dep(k_col_modes_r<N, true>, grid, smem_col_r<N>(), s, pdl, a, j0, mode);
            else
                launch_dep(k_col_modes_r<N, false>, grid, smem_col_r<N>(), s, pdl, a, j0, mode);
        } else if (a.bg && mode == COL_PROJECT)
            k_col_r<N, true, true><<<grid, kThreads, smem_col_r<N>(), s>>>(a, j0, mode);
        else if (a.bg)
            k_col_r<N, true, false><<<grid, kThreads, smem_col_r<N>(), s>>>(a, j0, mode);
        else if (mode == COL_PROJECT)
            launch_dep(k_col_r<N, false, true>, grid, smem_col_r<N>(), s, pdl, a, j0, mode);
        else
            launch_dep(k_col_r<N, false, false>, grid, smem_col_r<N>(), s, pdl, a, j0, mode);
        return;
    }
    dim3 grid(N / a.C2, nb);
    k_col<N><<<grid, kThreads, smem_col_t<N>(a.K, a.C2), s>>>(a, j0, mode);
}
template <int N>
void launch_row_bwd(const ProbArgs& a, int j0, int nb, int G, int mode, int upd_obj, int upd_probe, cudaStream_t s,
                    bool pdl) {
    if constexpr (has_reg<N>()) {
        dim3 grid(N / RegShape<N>::L, G * a.K);  // G frame slots per probe mode
        const size_t sm = smem_row_bwd_r<N>();
        if (mode != BWD_GRAD && upd_probe)  // AP and DM store Psi' alike
            launch_dep(k_row_bwd_r<N, 1>, grid, sm, s, pdl, a, j0, nb, mode, upd_obj, upd_probe);
        else if (mode == BWD_GRAD && upd_obj && !upd_probe)
            launch_dep(k_row_bwd_r<N, 2>, grid, sm, s, pdl, a, j0, nb, mode, upd_obj, upd_probe);
        else
            launch_dep(k_row_bwd_r<N, 0>, grid, sm, s, pdl, a, j0, nb, mode, upd_obj, upd_probe);
        return;
    }
    dim3 grid(N / a.L3, G);
    k_row_bwd<N><<<grid, kThreads, smem_row_bwd_t<N>(a.K, a.L3), s>>>(a, j0, nb, mode, upd_obj, upd_probe);
}
// Lines per block of the line-search kernels: 3 waves x L rows (columns) <= max_lines.
template <int N>
constexpr int ls_lines() {
    int L = 1;
    while (3 * L * 2 <= max_lines<N>() && N % (L * 2) == 0) L *= 2;
    return L;
}
template <int N>
void launch_row_fwd_ls(const ProbArgs& a, int j0, int nb, int pdl, cudaStream_t s) {
    if constexpr (has_reg<N>()) {
        if (a.K == 1) {
            dim3 grid(N / RegShape<N>::L, nb, (a.dir_obj && a.dir_probe) ? 3 : 2);
            launch_dep(k_row_fwd_ls_r<N>, grid, smem_row_fwd_r<N>(), s, pdl != 0, a, j0);
            return;
        }
    }
    constexpr int L = ls_lines<N>();
    dim3 grid(N / L, nb);
    k_row_fwd_ls<N><<<grid, kThreads, sizeof(float2) * (N + (size_t)3 * L * line_pitch<N>()), s>>>(a, j0, L);
}
template <int N>
void launch_col_ls(const ProbArgs& a, int j0, int nb, int pdl, cudaStream_t s) {
    if constexpr (has_reg<N>()) {
        if (a.K == 1) {
            dim3 grid(N / RegShape<N>::C, nb);
            launch_dep(k_col_ls_r<N>, grid, smem_col_r<N>(), s, pdl != 0, a, j0, (a.dir_obj && a.dir_probe) ? 3 : 2);
            return;
        }
    }
    constexpr int C = ls_lines<N>();
    dim3 grid(N / C, nb);
    const size_t sm = sizeof(float2) * (N + (size_t)3 * C * line_pitch<N>()) + sizeof(float) * 3 * (size_t)N * C;
    k_col_ls<N><<<grid, kThreads, sm, s>>>(a, j0, C);
}
template <int N>
void launch_fft2(float2* data, int nframes, int dir, cudaStream_t s) {
    constexpr int ml = max_lines<N>();
    int L = 1;
    while (L * 2 <= ml && N % (L * 2) == 0) L *= 2;
    size_t sm = sizeof(float2) * (N + (size_t)L * line_pitch<N>());
    dim3 grid(N / L, nframes);
    if (dir < 0) {
        k_fft_rows<N, -1><<<grid, kThreads, sm, s>>>(data, L);
        k_fft_cols<N, -1><<<grid, kThreads, sm, s>>>(data, L);
    } else {
        k_fft_rows<N, +1><<<grid, kThreads, sm, s>>>(data, L);
        k_fft_cols<N, +1><<<grid, kThreads, sm, s>>>(data, L);
    }
}

template <int N>
cudaError_t set_attrs_t() {
    cudaError_t e;
    const int mx = 200 * 1024;
    if ((e = cudaFuncSetAttribute(k_row_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_col<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_row_bwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_fft_rows<N, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_fft_rows<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_fft_cols<N, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_fft_cols<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_row_fwd_ls<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_col_ls<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if constexpr (has_reg<N>()) {
        if ((e = set_attrs_r<N>())) return e;
        if ((e = set_attrs_nf<N>())) return e;
    }
    return cudaSuccess;
}

// Resident row-backward blocks per SM from the occupancy calculator (cached
// once known; 0 while it cannot be asked, e.g. before the kernel attributes
// are set).
template <int N>
int row_bwd_per_sm() {
    static int v = 0;
    if (v == 0) {
        int n = 0;
        cudaError_t e;
        if constexpr (has_reg<N>())
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_row_bwd_r<N, 1>, kThreads, smem_row_bwd_r<N>());
        else
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_row_bwd<N>, kThreads,
                                                              smem_row_bwd_t<N>(1, max_lines<N>()));
        if (e != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        v = n;
    }
    return v;
}

template <int N>
const KernelSet* make_kernel_set() {
    constexpr int rl = has_reg<N>() ? reg_lines<N>() : 0;
    constexpr int rc = has_reg<N>() ? reg_cols<N>() : 0;
    static const KernelSet ks = {N,
                                 &launch_row_fwd<N>,
                                 &launch_col<N>,
                                 &launch_row_bwd<N>,
                                 &launch_fft2<N>,
                                 &launch_row_fwd_ls<N>,
                                 &launch_col_ls<N>,
                                 max_lines<N>(),
                                 ls_lines<N>(),
                                 rl,
                                 rc,
                                 &row_bwd_per_sm<N>,
                                 Plan<N>::R,
                                 Plan<N>::M,
                                 ColTma<N>::kOk ? &launch_col_tma<N> : nullptr,
                                 &col_tma_grid<N>,
                                 &launch_col_nf<N>,
                                 &launch_row_proj<N>};
    return &ks;
}

}  // namespace ptx
