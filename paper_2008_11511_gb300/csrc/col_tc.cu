// Column pass with the 16-point DFT stages on the tensor cores (the
// split-precision "chosen form"; one probe mode, N = 256 = 16 x 16).
//
// Each of the four DFT stages of a block's 256 column vectors (two forward,
// two inverse) is a real GEMM on the 5th-generation tensor cores:
//   D[256 x 32] = A[256 x 32] B^T,   A row v = vector v (16 complex, re/im
//   interleaved), B = the 32 x 32 real form of the 16-point DFT matrix,
// issued as tcgen05.mma kind::tf32 by one thread, operands in shared memory
// (K-major, 128-byte swizzled), accumulator in TMEM (2 x 128 lanes x 32
// columns), read back with tcgen05.ld.  FP32 accuracy comes from a hi + lo
// split of both operands (tf32 keeps 10 explicit mantissa bits; hi is the
// truncated value, lo = x - hi): A B ~ A_hi B_hi + A_lo B_hi + A_hi B_lo,
// about 2^-21 relative per product.  BF16 hi + lo (2^-16 per product) would
// leave the cycle above its 1e-5 tolerance after the eight stages of a
// cycle, so the split uses TF32.
//
// Vector v is owned by thread v: it writes row v of A for the first stage of
// each transform and reads row v of D (TMEM lane v % 128 of M-tile v / 128,
// warp v / 32 reading its lane quadrant).  Between the two stages of a
// transform the twiddle is applied in registers and the transpose is folded
// into the A writes of the next stage (thread (c, n1) writes element n1 of the
// vectors (c, k2)).  The projection and the LLK run in registers as in the
// FP32 column pass.
#include "kernels.cuh"

namespace ptx {

namespace tc {

constexpr int N = 256, C = 16;  // 16 columns per block, 256 threads
constexpr int kRow = 128;                        // bytes per A / B row (32 floats)
constexpr size_t kA = (size_t)256 * kRow;        // 32 KB per A part
constexpr size_t kB = (size_t)32 * kRow;         // 4 KB per B part
constexpr size_t kOffAhi = 0, kOffAlo = kOffAhi + kA;
constexpr size_t kOffB = kOffAlo + kA;           // fwd hi, fwd lo, inv hi, inv lo
constexpr size_t kOffTw = kOffB + 4 * kB;
constexpr size_t kOffBar = kOffTw + sizeof(float2) * N;
constexpr size_t kOffTmem = kOffBar + 8;
constexpr size_t kBytes = kOffTmem + 8 + 1024;   // + room to align the base to 1024
constexpr uint32_t kTmemCols = 64;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(16 >> 4) << 16;    // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}
// kind::tf32, D f32, A and B tf32 K-major, N = 32, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > (1ll << 31)) return false;
    }
}
// 32 consecutive fp32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// byte offset of float index k (0..31) of row r in a K-major 128-byte-swizzled tile
__device__ __forceinline__ uint32_t sw_off(int r, int k) {
    return (uint32_t)(r * kRow + ((((k >> 2) ^ (r & 7))) << 4) + ((k & 3) << 2));
}

}  // namespace tc

// grid (16, frames in batch), 256 threads; same arguments and outputs as k_col_r<256>.
__global__ void __launch_bounds__(256, 2) k_col_tc(ProbArgs a, int j0) {
    using namespace tc;
    extern __shared__ unsigned char smraw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* Ahi = sm + kOffAhi;
    unsigned char* Alo = sm + kOffAlo;
    unsigned char* Bm = sm + kOffB;
    float2* tw = (float2*)(sm + kOffTw);
    const uint32_t bar = su32(sm + kOffBar);
    uint32_t* tmem_slot = (uint32_t*)(sm + kOffTmem);
    __shared__ double red_s[8];
    const int t = threadIdx.x, warp = t >> 5;
    const int x0 = blockIdx.x * C;
    const int b = blockIdx.y;
    const int j = j0 + b;
    const int c = t % C, q = t / C;  // pass roles: (column c, n1 / k2 / kk = q)
    float2* spec = a.spec + (size_t)b * N * N + x0;

    // twiddles and the two DFT matrices in their real 32 x 32 form, split hi / lo
    load_twiddles<N>(tw);
    for (int e = t; e < 2 * 32 * 32; e += 256) {
        const int inv = e >> 10, n = (e >> 5) & 31, k = e & 31;
        const int kout = n >> 1, nin = k >> 1;
        float s, co;
        sincospif((inv ? 2.0f : -2.0f) * (float)((kout * nin) & 15) / 16.0f, &s, &co);
        // out re: Fr xr - Fi xi; out im: Fi xr + Fr xi
        const float v = (n & 1) == 0 ? ((k & 1) == 0 ? co : -s) : ((k & 1) == 0 ? s : co);
        const float hi = tf32_hi(v);
        unsigned char* base = Bm + (size_t)(2 * inv) * kB;
        *(float*)(base + sw_off(n, k)) = hi;
        *(float*)(base + kB + sw_off(n, k)) = v - hi;
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // this thread's D row: M-tile t / 128 at column 32 (t / 128), lane t % 128
    const uint32_t my_d = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (t >> 7));
    uint32_t parity = 0;

    // one tensor-core DFT stage over the A tile: D = A B^T, B = matrix `m` (0 fwd, 1 inv).
    // Every thread waits (bounded) for the stage's commit; the outcome is made
    // block-uniform, so a give-up seen by any thread stops the whole block: no
    // later stage issues MMAs, and the caller reports it and frees TMEM.
    auto stage = [&](int m, float* out) -> bool {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (t == 0) {
            const uint32_t bhi = su32(Bm + (size_t)(2 * m) * kB), blo = bhi + (uint32_t)kB;
#pragma unroll
            for (int tile = 0; tile < 2; ++tile) {
                const uint32_t ahi = su32(Ahi) + tile * 128 * kRow, alo = su32(Alo) + tile * 128 * kRow;
                const uint32_t d = tmem + 32 * tile;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    mma_tf32(d, desc_sw128(ahi + 32 * k), desc_sw128(bhi + 32 * k), k > 0);
                    mma_tf32(d, desc_sw128(alo + 32 * k), desc_sw128(bhi + 32 * k), 1);
                    mma_tf32(d, desc_sw128(ahi + 32 * k), desc_sw128(blo + 32 * k), 1);
                }
            }
            commit(bar);
        }
        const bool mine = bar_wait(bar, parity);
        if (__syncthreads_or(!mine)) return false;  // parity stays at the pending phase
        parity ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem_ld32(my_d, out);
        return true;
    };
    // write this thread's 16 complex values as its own A row (hi, lo)
    auto put_row = [&](const float2* v) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 x = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
            const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
            const uint32_t off = sw_off(t, 4 * i);
            *(float4*)(Ahi + off) = h;
            *(float4*)(Alo + off) = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
        }
    };
    // element `e` of the vectors (c, k) for k = 0..15 (rows k * 16 + c): the folded transpose
    auto put_col = [&](const float2* v, int e) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int r = k * 16 + c;
            const uint32_t off = sw_off(r, 2 * e);
            const float2 h = make_float2(tf32_hi(v[k].x), tf32_hi(v[k].y));
            *(float2*)(Ahi + off) = h;
            *(float2*)(Alo + off) = make_float2(v[k].x - h.x, v[k].y - h.y);
        }
    };

    float2 v[16];
    float o[32];
    // forward stage 1: vector (c, n1 = q) = x[q + 16 n2], n2 = 0..15
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) v[n2] = ld_hint(spec + (size_t)(q + 16 * n2) * N + c, policy_evict_last());
    // intensities and mask bits of the pass-2 pixels (rows q + 16 k1 of column c)
    float io[16];
    {
        const float* ib = a.iobs + (size_t)j * N * N + (size_t)q * N + x0 + c;
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) io[k1] = __ldcs(ib + (size_t)16 * k1 * N);
    }
    const uint32_t mbits = a.mbits[blockIdx.x * 256 + t];
    constexpr float invN2 = 1.0f / float(N * N);
    KahanF llk;
    put_row(v);
    // `good` is block-uniform (each stage combines the threads' wait outcomes)
    bool good = stage(0, o);
    if (good) {
        // twiddle w^(n1 k2) and the transpose into the vectors (c, k2)
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            const float2 y = make_float2(o[2 * k2], o[2 * k2 + 1]);
            v[k2] = k2 == 0 ? y : cmul(y, tw_get<N, -1>(tw, k2, q));
        }
        // the A tile may be rewritten at once: the stage's MMAs have completed (mbarrier);
        // the next stage's barrier orders every thread's D read before its MMAs
        put_col(v, q);
        good = stage(0, o);
    }
    if (good) {
        // projection and LLK on X^[q + 16 k1] (thread = vector (c, k2 = q))
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) {
            const float2 X = make_float2(o[2 * k1], o[2 * k1 + 1]);
            const float ic = cnorm(X) * invN2;
            const bool masked = (mbits >> k1) & 1u;
            if (!masked) llk.add(llk_term_fast(ic, io[k1]));
            const float f = masked ? 0.f : (amp_ratio(io[k1], ic) - 1.0f) * invN2;
            v[k1] = cscale(X, f);
        }
        // inverse stage 1 over k1 on the thread's own vector, then twiddle w^(+k2 kk)
        put_row(v);
        good = stage(1, o);
    }
    if (good) {
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const float2 y = make_float2(o[2 * kk], o[2 * kk + 1]);
            v[kk] = kk == 0 ? y : cmul(y, tw_get<N, +1>(tw, q, kk));
        }
        put_col(v, q);
        good = stage(1, o);
    }
    if (good) {
        // rows kk + 16 k1' of column c (thread = vector (c, kk = q))
        const uint64_t el = policy_evict_last();
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1)
            st_hint(spec + (size_t)(q + 16 * k1) * N + c, make_float2(o[2 * k1], o[2 * k1 + 1]), el);
    }
    const double tot = block_sum_double<256>(llk.value(), red_s);
    if (t == 0) {
        a.llk_part[(size_t)j * gridDim.x + blockIdx.x] = tot;
        if (!good) {
            // a stage's commit did not arrive in time: wait once more (bounded) for
            // the MMAs in flight before TMEM is freed, and report the give-up
            bar_wait(bar, parity);
            if (a.err_flag) {
                *(volatile int*)a.err_flag = 1;
                __threadfence_system();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

void launch_col_tc(const ProbArgs& a, int j0, int nb, cudaStream_t s) {
    dim3 grid(tc::N / tc::C, nb);
    k_col_tc<<<grid, 256, tc::kBytes, s>>>(a, j0);
}
cudaError_t set_attrs_tc() {
    cudaError_t e = cudaFuncSetAttribute(k_col_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::kBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_col_tc, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
}

}  // namespace ptx
