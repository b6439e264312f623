// Near-field passes (PropagateNearField, one probe mode).
//
// In the near field the detector sees the exit wave after a paraxial Fresnel
// propagation, IFT(FT(X) h), h[ky][kx] = t[ky] t[kx], t[k] = exp(-i pi c k^2 / N^2)
// (k signed, c = lambda z / pixel^2), and the amplitude projection acts on
// that propagated wave in detector pixels.  The cycle of a batch becomes five
// passes through the Fourier work stack:
//
//   row_fwd   (shared with the far field)  X -> row FFT
//   col_nf +1 column FFT, x h / N^2, inverse column FFT
//   row_proj  inverse row FFT -> detector wave; projection + LLK giving the
//             correction (s - 1) Psi_det; row FFT
//   col_nf -1 column FFT, x conj(h) / N^2, inverse column FFT
//   row_bwd   (shared) inverse row FFT -> D; Psi' = Phi + D; probe sums
//
// so D = Prop^-1((s - 1) Prop(X)), as in the far field with Prop for FT.
#pragma once
#include "kernels_reg.cuh"

namespace ptx {

// ---------------------------------------------------------------------------
// Column pass of the propagator: grid (N / L, frames in batch); block
// handles columns [x0, x0 + L).  nf_t = t[k] (complex64, k in FFT order).
// ---------------------------------------------------------------------------
template <int N, int DIR>
__global__ void __launch_bounds__(kThreads, RegShape<N>::ColMinBlocks) k_col_nf(ProbArgs a) {
    using S = RegShape<N>;
    constexpr int R = S::R, M = S::M, C = S::L, P = S::P;
    constexpr int I1b = (C * M + kThreads - 1) / kThreads;
    extern __shared__ __align__(16) float2 sm[];
    float2* tw = sm;
    float2* buf = sm + N;
    load_twiddles<N>(tw);
    const int x0 = blockIdx.x * C;
    const int b = blockIdx.y;
    float2* spec = a.spec + (size_t)b * N * N + x0;
    __syncthreads();
    // forward pass 1: thread (c, n1) holds rows n1 + M n2 of column c
#pragma unroll
    for (int i = 0; i < S::I1; ++i) {
        const int w = threadIdx.x + i * kThreads;
        if (w < C * M) {
            const int n1 = w / C, c = w - n1 * C;
            float2 v[R];
#pragma unroll
            for (int n2 = 0; n2 < R; ++n2) v[n2] = spec[(size_t)(n1 + M * n2) * N + c];
            Dft<R, -1>::run(v);
            float2* o = buf + c * P + n1;
            o[0] = v[0];
#pragma unroll
            for (int k2 = 1; k2 < R; ++k2) o[k2 * (M + 1)] = cmul(v[k2], tw_get<N, -1>(tw, k2, n1));
        }
    }
    __syncthreads();
    float2 u[S::I2][M];
#pragma unroll
    for (int i = 0; i < S::I2; ++i) {
        const int w = threadIdx.x + i * kThreads;
        if (w < C * R) {
            const int k2 = w / C, c = w - k2 * C;
            const float2* src = buf + c * P + k2 * (M + 1);
#pragma unroll
            for (int n1 = 0; n1 < M; ++n1) u[i][n1] = src[n1];
        }
    }
    __syncthreads();
    constexpr float invN2 = 1.0f / float(N * N);
#pragma unroll
    for (int i = 0; i < S::I2; ++i) {
        const int w = threadIdx.x + i * kThreads;
        if (w < C * R) {
            const int k2 = w / C, c = w - k2 * C;
            Dft<M, -1>::run(u[i]);
            // X^[ky = k2 + R k1][kx] times h (or conj(h)) / N^2
            float2 tx = a.nf_t[x0 + c];
            if constexpr (DIR < 0) tx.y = -tx.y;
#pragma unroll
            for (int k1 = 0; k1 < M; ++k1) {
                float2 ty = a.nf_t[k2 + R * k1];
                if constexpr (DIR < 0) ty.y = -ty.y;
                u[i][k1] = cscale(cmul(u[i][k1], cmul(ty, tx)), invN2);
            }
            Dft<M, +1>::run(u[i]);
            float2* o = buf + c * P + k2;
            o[0] = u[i][0];
#pragma unroll
            for (int kk = 1; kk < M; ++kk) o[kk * (R + 1)] = cmul(u[i][kk], tw_get<N, +1>(tw, k2, kk));
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
#pragma unroll
            for (int k1 = 0; k1 < R; ++k1) spec[(size_t)(kk + M * k1) * N + c] = v[k1];
        }
    }
}

// ---------------------------------------------------------------------------
// Row pass at the detector: inverse row FFT of the propagated rows gives the
// detector wave; per pixel I_c = |Psi_det|^2, the Poisson LLK term and the
// correction (s - 1) Psi_det (0 where masked); then the row FFT of the
// correction back into the work stack (skipped with llk_only).
// grid (N / L, frames in batch); block handles rows [y0, y0 + L) of frame j0 + blockIdx.y.
// ---------------------------------------------------------------------------
// kCycle: the cycle's form (the correction written back, no background) fixed
// at compile time; otherwise llk_only and the background come from the arguments.
template <int N, bool kCycle>
__global__ void __launch_bounds__(kThreads, RegShape<N>::ColMinBlocks) k_row_proj(ProbArgs a, int j0, int llk_only_arg) {
    const int llk_only = kCycle ? 0 : llk_only_arg;
    const float* bgp = kCycle ? nullptr : a.bg;
    using S = RegShape<N>;
    constexpr int R = S::R, M = S::M, L = S::L, P = S::P;
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red_s[kThreads / 32];
    float2* tw = sm;
    float2* buf = sm + N;
    load_twiddles<N>(tw);
    const int y0 = blockIdx.x * L;
    const int b = blockIdx.y;
    const int j = j0 + b;
    float2* spec = a.spec + ((size_t)b * N + y0) * N;
    __syncthreads();
    // inverse pass 1: thread (line, n1) holds elements n1 + M n2 of its row
#pragma unroll
    for (int i = 0; i < S::I1; ++i) {
        const int w = threadIdx.x + i * kThreads;
        if (w < L * M) {
            const int line = w / M, n1 = w - line * M;
            float2 v[R];
#pragma unroll
            for (int n2 = 0; n2 < R; ++n2) v[n2] = spec[(size_t)line * N + n1 + M * n2];
            Dft<R, +1>::run(v);
            float2* o = buf + line * P + n1;
            o[0] = v[0];
#pragma unroll
            for (int k2 = 1; k2 < R; ++k2) o[k2 * (M + 1)] = cmul(v[k2], tw_get<N, +1>(tw, k2, n1));
        }
    }
    __syncthreads();
    // inverse pass 2: thread (line, k2) holds the detector wave at x = k2 + R k1
    float2 u[S::I2][M];
#pragma unroll
    for (int i = 0; i < S::I2; ++i) {
        const int w = threadIdx.x + i * kThreads;
        if (w < L * R) {
            const int line = w / R, k2 = w - line * R;
            const float2* src = buf + line * P + k2 * (M + 1);
#pragma unroll
            for (int n1 = 0; n1 < M; ++n1) u[i][n1] = src[n1];
        }
    }
    __syncthreads();
    float llk = 0.f;  // the terms are >= 0: a plain float sum of a thread's pixels
#pragma unroll
    for (int i = 0; i < S::I2; ++i) {
        const int w = threadIdx.x + i * kThreads;
        if (w < L * R) {
            const int line = w / R, k2 = w - line * R;
            const int y = y0 + line;
            Dft<M, +1>::run(u[i]);
            const float* io_row = a.iobs + ((size_t)j * N + y) * N + k2;
            const uint8_t* mk_row = a.mask + (size_t)y * N + k2;
#pragma unroll
            for (int k1 = 0; k1 < M; ++k1) {
                float ic = cnorm(u[i][k1]);
                const float io = __ldcs(io_row + R * k1);
                const bool masked = mk_row[R * k1] != 0;
                if (bgp) {  // incoherent background in the detector plane
                    const int pix = y * N + k2 + R * k1;
                    ic += __ldg(bgp + pix);
                    if (a.bg_acc && !masked) atomicAdd(a.bg_acc + pix, fmaxf(io, 0.f) / fmaxf(ic, 1e-30f));
                }
                if (!masked) llk += llk_term_fast(ic, io);
                const float f = masked ? 0.f : amp_ratio(io, ic) - 1.0f;
                u[i][k1] = cscale(u[i][k1], f);
            }
            if (!llk_only) {
                // the correction in natural order, for the forward row FFT
                float2* o = buf + line * P + k2;
#pragma unroll
                for (int k1 = 0; k1 < M; ++k1) o[R * k1] = u[i][k1];
            }
        }
    }
    const double tot = block_sum_double<kThreads>((double)llk, red_s);
    if (threadIdx.x == 0) a.llk_part[(size_t)j * gridDim.x + blockIdx.x] = tot;
    if (llk_only) return;
    __syncthreads();
    // forward pass 1 from the natural-order correction: thread (line, n1)
    float2 v[S::I1][R];
#pragma unroll
    for (int i = 0; i < S::I1; ++i) {
        const int w = threadIdx.x + i * kThreads;
        if (w < L * M) {
            const int line = w / M, n1 = w - line * M;
            const float2* src = buf + line * P + n1;
#pragma unroll
            for (int n2 = 0; n2 < R; ++n2) v[i][n2] = src[M * n2];
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < S::I1; ++i) {
        const int w = threadIdx.x + i * kThreads;
        if (w < L * M) {
            const int line = w / M, n1 = w - line * M;
            Dft<R, -1>::run(v[i]);
            float2* o = buf + line * P + n1;
            o[0] = v[i][0];
#pragma unroll
            for (int k2 = 1; k2 < R; ++k2) o[k2 * (M + 1)] = cmul(v[i][k2], tw_get<N, -1>(tw, k2, n1));
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < S::I2; ++i) {
        const int w = threadIdx.x + i * kThreads;
        if (w < L * R) {
            const int line = w / R, k2 = w - line * R;
            float2 t[M];
            const float2* src = buf + line * P + k2 * (M + 1);
#pragma unroll
            for (int n1 = 0; n1 < M; ++n1) t[n1] = src[n1];
            Dft<M, -1>::run(t);
            float2* dst = spec + (size_t)line * N + k2;
#pragma unroll
            for (int k1 = 0; k1 < M; ++k1) dst[R * k1] = t[k1];
        }
    }
}

template <int N>
size_t smem_nf() {
    using S = RegShape<N>;
    return sizeof(float2) * (N + (size_t)S::L * S::P);
}

template <int N>
void launch_col_nf(const ProbArgs& a, int nb, int dir, cudaStream_t s) {
    if constexpr (Plan<N>::M > 1) {
        dim3 grid(N / RegShape<N>::L, nb);
        if (dir < 0)
            k_col_nf<N, -1><<<grid, kThreads, smem_nf<N>(), s>>>(a);
        else
            k_col_nf<N, +1><<<grid, kThreads, smem_nf<N>(), s>>>(a);
    }
}
template <int N>
void launch_row_proj(const ProbArgs& a, int j0, int nb, int llk_only, cudaStream_t s) {
    if constexpr (Plan<N>::M > 1) {
        dim3 grid(N / RegShape<N>::L, nb);
        if (!llk_only && !a.bg)
            k_row_proj<N, true><<<grid, kThreads, smem_nf<N>(), s>>>(a, j0, llk_only);
        else
            k_row_proj<N, false><<<grid, kThreads, smem_nf<N>(), s>>>(a, j0, llk_only);
    }
}
template <int N, class F>
cudaError_t nf_attrs(F f) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
}
template <int N>
cudaError_t set_attrs_nf() {
    if constexpr (Plan<N>::M > 1) {
        cudaError_t e;
        if ((e = nf_attrs<N>(k_col_nf<N, -1>))) return e;
        if ((e = nf_attrs<N>(k_col_nf<N, +1>))) return e;
        if ((e = nf_attrs<N>(k_row_proj<N, true>))) return e;
        if ((e = nf_attrs<N>(k_row_proj<N, false>))) return e;
    }
    return cudaSuccess;
}

}  // namespace ptx
