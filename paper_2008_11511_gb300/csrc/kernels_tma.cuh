// Column pass fed by the tensor memory accelerator (one probe mode).
//
// A persistent grid walks the batch's (frame, column block) items.  Each
// item's input — the block's C columns of the Fourier work stack (N rows x C
// complex values) and the same columns of the measured intensities — arrives
// in shared memory by two 2D tensor copies (cp.async.bulk.tensor) that
// complete on an mbarrier.  The copy for the CTA's next item is issued as soon
// as the current item's inputs have been read into registers, so it overlaps
// the rest of the item: the transforms never wait on L2 or HBM.  The
// arithmetic is that of the register column pass: forward column FFT,
// amplitude projection and Poisson LLK, inverse column FFT of the correction.
#pragma once
#include <cuda.h>

#include "kernels_reg.cuh"

namespace ptx {

namespace tma {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity for at most ~2^31 SM clocks (about a
// second at the GB300 clock); false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1ll << 31)) return false;
    return true;
}
// Generic-proxy accesses to shared memory before async-proxy writes to it.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 2D tiled tensor copy global -> shared, completing on `bar`, with an L2 policy.
__device__ __forceinline__ void load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar,
                                        uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void report(int* flag) {
    if (flag) {
        *(volatile int*)flag = 1;
        __threadfence_system();
    }
}

}  // namespace tma

// Shared-memory layout of k_col_t (bytes, in order): spec tile [N][C] float2,
// intensity tile [N][C] float, mask tile [N][C] uint8, transpose buffer [C][P]
// float2, twiddles [N], mbarrier.
template <int N>
struct ColTma {
    static constexpr int R = Plan<N>::R, M = Plan<N>::M, C = reg_lines<N>(), P = reg_pitch<N>(), XB = N / C;
    static constexpr size_t kSpec = 0;
    static constexpr size_t kIo = kSpec + sizeof(float2) * N * C;
    static constexpr size_t kMask = kIo + sizeof(float) * N * C;
    static constexpr size_t kBuf = kMask + (size_t)N * C;
    static constexpr size_t kTw = kBuf + sizeof(float2) * C * P;
    static constexpr size_t kBar = kTw + sizeof(float2) * N;
    static constexpr size_t kBytes = kBar + 8;
    static constexpr uint32_t kTx = (uint32_t)((sizeof(float2) + sizeof(float) + 1) * N * C);
    // one pass-1 item and one pass-2 item per thread, a tensor box of at most 256 rows
    static constexpr bool kOk = M > 1 && C * M == kThreads && C * R == kThreads && N <= 256 && M <= 16;
};

// grid: persistent (a multiple of the SMs); items b * XB + xb for frames
// j0 + b, b < nb, column blocks xb.  tm_spec maps the lane's work stack as
// [nb * N rows][N] 8-byte elements, tm_io the intensities as [J * N][N] floats,
// tm_mask the detector mask as [N][N] bytes.
template <int N>
__global__ void __launch_bounds__(kThreads, 2)
    k_col_t(const __grid_constant__ CUtensorMap tm_spec, const __grid_constant__ CUtensorMap tm_io,
            const __grid_constant__ CUtensorMap tm_mask, ProbArgs a, int j0, int nb) {
    using L = ColTma<N>;
    constexpr int R = L::R, M = L::M, C = L::C, P = L::P, XB = L::XB;
    static_assert(L::kOk, "one item per thread in both passes");
    extern __shared__ __align__(128) unsigned char smt[];
    unsigned char* sm = smt;
    float2* st_spec = (float2*)(sm + L::kSpec);
    float* st_io = (float*)(sm + L::kIo);
    float2* buf = (float2*)(sm + L::kBuf);
    float2* tw = (float2*)(sm + L::kTw);
    uint8_t* st_mask = sm + L::kMask;
    __shared__ double red_s[kThreads / 32];
    const uint32_t bar = tma::smem_u32(sm + L::kBar);
    const int t = threadIdx.x;
    // pass-1 role (column c, rows n1 + M n2) and pass-2 role (column c, rows k2 + R k1)
    const int c = t % C, q = t / C;

    load_twiddles<N>(tw);
    if (t == 0) {
        tma::mbar_init(bar, 1);
        tma::fence_mbar_init();
    }
    __syncthreads();

    const int nitems = nb * XB;
    auto issue = [&](int it) {
        const int b = it / XB, xb = it - b * XB;
        tma::mbar_expect_tx(bar, L::kTx);
        tma::load_2d(tma::smem_u32(st_spec), &tm_spec, xb * C, b * N, bar, policy_evict_last());
        tma::load_2d(tma::smem_u32(st_io), &tm_io, xb * C, (j0 + b) * N, bar, policy_evict_first());
        tma::load_2d(tma::smem_u32(st_mask), &tm_mask, xb * C, 0, bar, policy_evict_last());
    };
    if (t == 0 && (int)blockIdx.x < nitems) issue(blockIdx.x);
    uint32_t parity = 0;
    constexpr float invN2 = 1.0f / float(N * N);

    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int b = it / XB, xb = it - b * XB;
        const int x0 = xb * C;
        const bool late = !tma::mbar_wait_bounded(bar, parity);
        parity ^= 1u;
        // forward pass 1 from the staged tile: thread (c, n1 = q) holds rows q + M n2
        float io[M];
        uint32_t mbits = 0u;
        {
            float2 v[R];
#pragma unroll
            for (int n2 = 0; n2 < R; ++n2) v[n2] = st_spec[(q + M * n2) * C + c];
#pragma unroll
            for (int k1 = 0; k1 < M; ++k1) {
                io[k1] = st_io[(q + R * k1) * C + c];
                mbits |= st_mask[(q + R * k1) * C + c] ? (1u << k1) : 0u;
            }
            Dft<R, -1>::run(v);
            float2* o = buf + c * P + q;
            o[0] = v[0];
#pragma unroll
            for (int k2 = 1; k2 < R; ++k2) o[k2 * (M + 1)] = cmul(v[k2], tw_get<N, -1>(tw, k2, q));
        }
        // the tile is consumed: the next item's copy overlaps the rest of this one
        if (__syncthreads_or(late)) {
            if (t == 0) {
                tma::report(a.err_flag);
                tma::mbar_wait_bounded(bar, parity ^ 1u);  // the copy that was late, if it still lands
            }
            return;
        }
        if (t == 0 && it + (int)gridDim.x < nitems) {
            tma::fence_proxy_async();
            issue(it + gridDim.x);
        }
        // forward pass 2: thread (c, k2 = q) holds X^[q + R k1]
        float2 u[M];
        {
            const float2* src = buf + c * P + q * (M + 1);
#pragma unroll
            for (int n1 = 0; n1 < M; ++n1) u[n1] = src[n1];
        }
        __syncthreads();
        KahanF llk;
        Dft<M, -1>::run(u);
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) {
            const float ic = cnorm(u[k1]) * invN2;
            const bool masked = (mbits >> k1) & 1u;
            if (!masked) llk.add(llk_term_fast(ic, io[k1]));
            const float f = masked ? 0.f : (amp_ratio(io[k1], ic) - 1.0f) * invN2;
            u[k1] = cscale(u[k1], f);
        }
        // inverse pass 1: M-point codelet over k1, twiddle, y'[k2' (R+1) + k2]
        Dft<M, +1>::run(u);
        {
            float2* o = buf + c * P + q;
            o[0] = u[0];
#pragma unroll
            for (int kk = 1; kk < M; ++kk) o[kk * (R + 1)] = cmul(u[kk], tw_get<N, +1>(tw, q, kk));
        }
        const double tot = block_sum_double<kThreads>(llk.value(), red_s);
        if (t == 0) a.llk_part[(size_t)(j0 + b) * XB + xb] = tot;
        __syncthreads();
        // inverse pass 2: thread (c, k2' = q) reads y'[q (R+1) + n], R-point codelet, rows q + M k1'
        {
            float2 v[R];
            const float2* src = buf + c * P + q * (R + 1);
#pragma unroll
            for (int n = 0; n < R; ++n) v[n] = src[n];
            Dft<R, +1>::run(v);
            float2* spec = a.spec + (size_t)b * N * N + x0;
            const uint64_t el = policy_evict_last();
#pragma unroll
            for (int k1 = 0; k1 < R; ++k1) st_hint(spec + (size_t)(q + M * k1) * N + c, v[k1], el);
        }
        __syncthreads();  // buf is rewritten by the next item
    }
}

template <int N>
void launch_col_tma(const void* tm_spec, const void* tm_io, const void* tm_mask, const ProbArgs& a, int j0, int nb,
                    int grid, cudaStream_t s) {
    if constexpr (ColTma<N>::kOk) {
        const int nitems = nb * ColTma<N>::XB;
        if (grid > nitems) grid = nitems;
        k_col_t<N><<<grid, kThreads, ColTma<N>::kBytes, s>>>(
            *(const CUtensorMap*)tm_spec, *(const CUtensorMap*)tm_io, *(const CUtensorMap*)tm_mask, a, j0, nb);
    }
}

// Resident CTAs of k_col_t over the whole GPU (0: not available for N).
template <int N>
int col_tma_grid() {
    if constexpr (ColTma<N>::kOk) {
        static int g = -1;
        if (g >= 0) return g;
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaFuncSetAttribute(k_col_t<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ColTma<N>::kBytes) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_col_t<N>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_col_t<N>, kThreads, ColTma<N>::kBytes) !=
                cudaSuccess) {
            cudaGetLastError();
            return g = 0;
        }
        return g = per * sms;
    } else {
        return 0;
    }
}

}  // namespace ptx
