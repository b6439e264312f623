// Column pass with the 16-point DFT stages on the tensor cores (the
// split-precision form of the DFT stages; one probe mode, N = 256 = 16 x 16).
//
// Each of the four DFT stages of a block's 256 column vectors (two forward,
// two inverse) is a real GEMM on the 5th-generation tensor cores, one per
// half of the block (128 vectors of 8 columns):
//   D[128 x 32] = A[128 x 32] B^T,   A row v = vector v (16 complex, re/im
//   interleaved), B = the 32 x 32 real form of the 16-point DFT matrix,
// issued by one thread of the half, operands in shared memory (K-major,
// swizzled), accumulator in TMEM (128 lanes x 32 columns per half, FP32), read
// back with tcgen05.ld.  FP32 accuracy comes from splitting both operands into terms of
// the narrow type and summing the products of the terms that matter:
//
//   TF32X2  (kind::tf32): x = hi + lo, hi = x truncated to TF32 (10 explicit
//           mantissa bits), lo = x - hi; A B ~ Ah Bh + Al Bh + Ah Bl, about
//           2^-21 relative per product (3 products).
//   BF16X3  (kind::f16, bf16): x = hi + mid + lo, each the round-to-nearest
//           bf16 of what the previous terms leave; A B ~ Ah Bh + Ah Bm + Am Bh
//           + Ah Bl + Am Bm + Al Bh, the terms down to 2^-16 kept (6 products).
//   BF16X2  (kind::f16, bf16): x = hi + lo, A B ~ Ah Bh + Ah Bl + Al Bh
//           (3 products), about 2^-16 relative per product: the two-term
//           split, kept to measure its accuracy.
//
// Row u of a half's tile is owned by thread u of the half: it writes row u of
// A for the first stage of each transform and reads row u of D (TMEM lane u,
// warp u / 32 of the half reading its lane quadrant).  Between the two stages
// of a transform the twiddle is applied in registers and the transpose is
// folded into the A writes of the next stage (thread (c, n1) writes element n1
// of the vectors (c, k2), all in its own half).  The two halves synchronise
// only at each frame's LLK reduction, so within a frame one half's MMAs
// overlap the other half's SIMT work.  A block loops over about nb / 19
// frames with the matrices, twiddles and TMEM set up once.  The projection
// and the LLK run in registers as in the FP32 column pass.
#include <algorithm>

#include "tc.cuh"

namespace ptx {

// grid (16, frames in batch), 256 threads; same arguments and outputs as k_col_r<256>.
// The block's 16 columns form two independent halves (threads 128 h .. 128 h +
// 127, columns 8 h .. 8 h + 7), each with its own A tile, mbarrier, TMEM columns
// and named barrier (tc::Pipe256), so that one half's MMAs run while the other
// half splits, twiddles and stores.  Thread u = t % 128 of half h is (column
// c = 8 h + u % 8, q = u / 8) and owns row u of its half's tile in every stage;
// the stage-2 vectors (c, k) are rows 8 k + u % 8.
// selftest != 0: half 0 of block (0, 0) issues neither the MMAs nor the commit
// of its first stage, so that stage's bounded wait runs out with nothing in
// flight (the give-up path, exercised without a fault).
template <int F>
__global__ void __launch_bounds__(256, 2) k_col_tc(ProbArgs a, int j0, int nb, int selftest) {
    using namespace tc;
    extern __shared__ unsigned char smraw[];
    __shared__ double red_s[8];
    const int t = threadIdx.x;
    const int h = t >> 7, u = t & 127, cl = u & 7, q = u >> 3, c = 8 * h + cl;
    const int x0 = blockIdx.x * C;
    Pipe256<F> pp;
    pp.setup(smraw, selftest != 0 && blockIdx.x == 0 && blockIdx.y == 0 && h == 0);
    const float2* tw = pp.tw;

    float2 v[16];
    float o[32];
    bool good = true, bad = false;
    // mask bits of the thread's stage-2 pixels (the same for every frame); the
    // table is laid out for the FP32 column pass's threads (k2 * 16 + c)
    const uint32_t mbits = a.mbits[blockIdx.x * 256 + q * 16 + c];
    constexpr float invN2 = 1.0f / float(N * N);
    for (int b = blockIdx.y; b < nb; b += gridDim.y) {
        const int j = j0 + b;
        float2* spec = a.spec + (size_t)b * N * N + x0;
        // forward stage 1: vector (c, n1 = q) = x[q + 16 n2], n2 = 0..15
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) v[n2] = ld_hint(spec + (size_t)(q + 16 * n2) * N + c, policy_evict_last());
        // intensities of the stage-2 pixels (rows q + 16 k1 of column c)
        float io[16];
        {
            const float* ib = a.iobs + (size_t)j * N * N + (size_t)q * N + x0 + c;
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) io[k1] = __ldcs(ib + (size_t)16 * k1 * N);
        }
        float llk = 0.f;  // the terms are >= 0: a plain float sum of a thread's pixels
        pp.put_row(v);
        // `good` is uniform over the half (each stage combines its threads' wait outcomes)
        good = pp.stage(0, o);
        if (good) {
            // twiddle w^(n1 k2) and the transpose into the vectors (c, k2)
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) {
                const float2 y = make_float2(o[2 * k2], o[2 * k2 + 1]);
                v[k2] = k2 == 0 ? y : cmul(y, tw_get<N, -1>(tw, k2, q));
            }
            // the A tile may be rewritten at once: the stage's MMAs have completed (mbarrier);
            // the next stage's barrier orders every thread's D read before its MMAs
            pp.template put_col<8>(v, cl, q);
            good = pp.stage(0, o);
        }
        if (good) {
            // projection and LLK on X^[q + 16 k1] (thread = vector (c, k2 = q))
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                const float2 X = make_float2(o[2 * k1], o[2 * k1 + 1]);
                const float ic = cnorm(X) * invN2;
                const bool masked = (mbits >> k1) & 1u;
                float ratio;
                const float term = llk_term_ratio(ic, io[k1], ratio);
                if (!masked) llk += term;
                const float f = masked ? 0.f : (ratio - 1.0f) * invN2;
                v[k1] = cscale(X, f);
            }
            // inverse stage 1 over k1 on the thread's own vector, then twiddle w^(+k2 kk)
            pp.put_row(v);
            good = pp.stage(1, o);
        }
        if (good) {
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const float2 y = make_float2(o[2 * kk], o[2 * kk + 1]);
                v[kk] = kk == 0 ? y : cmul(y, tw_get<N, +1>(tw, q, kk));
            }
            pp.template put_col<8>(v, cl, q);
            good = pp.stage(1, o);
        }
        if (good) {
            // rows kk + 16 k1' of column c (thread = vector (c, kk = q))
            const uint64_t el = policy_evict_last();
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1)
                st_hint(spec + (size_t)(q + 16 * k1) * N + c, make_float2(o[2 * k1], o[2 * k1 + 1]), el);
        }
        const double tot = block_sum_pos<256>(llk, red_s);
        if (t == 0) a.llk_part[(size_t)j * gridDim.x + blockIdx.x] = tot;
        bad = __syncthreads_or(!good);  // also orders thread 0's reads of red_s before the next frame
        if (bad) break;
    }
    pp.finish(good, bad, a.err_flag);
}

// ---------------------------------------------------------------------------
// The 512-point column transforms on the tensor cores, any number of probe
// modes.  512 = 16 x 32: x[n1 + 32 n2] (n1 < 32, n2 < 16).
//   stage A (16-point DFT over n2): 512 vectors (c, n1) of the block's 16
//     columns, D[512 x 32] = A[512 x 32] B16^T (four 128-row tiles);
//   twiddle w_512^(n1 k2) in registers;
//   stage B (32-point DFT over n1): 256 vectors (c, k2), D[256 x 64] =
//     A[256 x 64] B32^T (two 128-row tiles, N = 64, K = 64 stored as two
//     K-planes of 32 elements, each a swizzled K-major tile);
//   X[k2 + 16 k1].  The inverse runs the same stages in the other order.
// Thread t (512 per block) owns stage-A vector t = (c = t % 16, n1 = t / 16)
// and reads row t of D; in stage B it reads half h = t / 256 (outputs
// 16 h .. 16 h + 15) of row r = t % 256 = (k2 = r / 16, c = r % 16).  The modes
// take two sweeps as in the FP32 multi-mode column pass: the forward
// transforms of every mode (X^_k written back to the work stack at the
// thread's own pixels, sum_k |X^_k|^2 kept in registers), then per pixel the
// common factor and the LLK, then per mode the reload, scale and inverse.
// ---------------------------------------------------------------------------

template <int F>
__global__ void __launch_bounds__(512, 1) k_col_tc512(ProbArgs a, int j0) {
    using namespace tc;
    constexpr int N = 512, C = 16;
    extern __shared__ unsigned char smraw[];
    __shared__ double red_s[16];
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * C;
    const int b = blockIdx.y;
    const int j = j0 + b;
    const int K = a.K;
    const int c1 = t % C, n1 = t / C;            // stage-A vector (column, n1); also (column, kk) at the end
    const int r2 = t & 255, h = t >> 8;          // stage-B row and half
    const int k2 = r2 / C, c2 = r2 % C;
    Pipe512<F> pp;
    pp.setup(smraw);
    const float2* tw = pp.tw;

    constexpr float invN2 = 1.0f / float(N * N);
    float2 v[16];
    float o[32];
    float ic[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) ic[i] = 0.f;
    bool good = true;
    // sweep 1: forward transforms of every mode; pixels rows k2 + 16 k1, k1 = 16 h + i, column c2
    for (int k = 0; k < K && good; ++k) {
        float2* spec = a.spec + ((size_t)b * K + k) * N * N + x0;
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) v[n2] = ld_hint(spec + (size_t)(n1 + 32 * n2) * N + c1, policy_evict_last());
#pragma unroll
        for (int i = 0; i < 16; ++i) pp.put(0, t, i, v[i]);  // stage-A row t
        good = pp.stage(false, 0, o);
        if (!good) break;
        // twiddle w^(n1 k2) and the transpose into the stage-B rows (k2, c)
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const float2 y = make_float2(o[2 * kk], o[2 * kk + 1]);
            const float2 yt = kk == 0 ? y : cmul(y, tw_get<N, -1>(tw, kk, n1));
            pp.put(n1 >> 4, kk * C + c1, n1 & 15, yt);
        }
        good = pp.stage(true, 0, o);
        if (!good) break;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float2 X = make_float2(o[2 * i], o[2 * i + 1]);
            ic[i] = fmaf(X.x, X.x, fmaf(X.y, X.y, ic[i]));
            if (K > 1) spec[(size_t)(k2 + 16 * (16 * h + i)) * N + c2] = X;  // this thread's own pixels
            v[i] = X;
        }
    }
    // the common factor and the LLK of the thread's 16 pixels
    KahanF llk;
    if (good) {
        const float* ib = a.iobs + (size_t)j * N * N + x0 + c2;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int row = k2 + 16 * (16 * h + i);
            const float io = __ldcs(ib + (size_t)row * N);
            const bool masked = a.mask[(size_t)row * N + x0 + c2] != 0;
            float ratio;
            const float term = llk_term_ratio(ic[i] * invN2, io, ratio);
            if (!masked) llk.add(term);
            ic[i] = masked ? 0.f : (ratio - 1.0f) * invN2;  // now the factor
        }
    }
    // sweep 2: per mode, the scaled spectrum through the inverse stages
    for (int k = 0; k < K && good; ++k) {
        float2* spec = a.spec + ((size_t)b * K + k) * N * N + x0;
        if (K > 1) {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = spec[(size_t)(k2 + 16 * (16 * h + i)) * N + c2];
        }
        // stage-B row r2, half h: elements k1 = 16 h + i
#pragma unroll
        for (int i = 0; i < 16; ++i) pp.put(h, r2, i, cscale(v[i], ic[i]));
        good = pp.stage(true, 1, o);
        if (!good) break;
        // twiddle w^(+k2 kk), kk = 16 h + i, and the transpose into the stage-A rows (kk, c)
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int kk = 16 * h + i;
            const float2 y = make_float2(o[2 * i], o[2 * i + 1]);
            pp.put(0, kk * C + c2, k2, (k2 == 0 || kk == 0) ? y : cmul(y, tw_get<N, +1>(tw, k2, kk)));
        }
        good = pp.stage(false, 1, o);
        if (!good) break;
        // rows kk + 32 k1' of column c (thread = stage-A row t = (c1, kk = n1))
        const uint64_t el = policy_evict_last();
#pragma unroll
        for (int i = 0; i < 16; ++i)
            st_hint(spec + (size_t)(n1 + 32 * i) * N + c1, make_float2(o[2 * i], o[2 * i + 1]), el);
    }
    const double tot = block_sum_double<512>(llk.value(), red_s);
    if (t == 0) a.llk_part[(size_t)j * gridDim.x + blockIdx.x] = tot;
    pp.finish(good, a.err_flag);
}

void launch_col_tc(const ProbArgs& a, int j0, int nb, int form, int selftest, cudaStream_t s) {
    if (a.N == 512) {
        dim3 grid(512 / 16, nb);
        if (form == TC_BF16X3)
            k_col_tc512<TC_BF16X3><<<grid, 512, tc::Fmt512<TC_BF16X3>::kBytes, s>>>(a, j0);
        else if (form == TC_BF16X2)
            k_col_tc512<TC_BF16X2><<<grid, 512, tc::Fmt512<TC_BF16X2>::kBytes, s>>>(a, j0);
        else
            k_col_tc512<TC_TF32X2><<<grid, 512, tc::Fmt512<TC_TF32X2>::kBytes, s>>>(a, j0);
        return;
    }
    // two blocks per SM; each block runs its 16 columns of about nb / G frames
    // (the matrices, twiddles and TMEM set up once per block)
    const int slots = std::max(1, 2 * sm_count() / (tc::N / tc::C));
    const int per = (nb + slots - 1) / slots;
    dim3 grid(tc::N / tc::C, (nb + per - 1) / per);
    if (form == TC_BF16X3)
        k_col_tc<TC_BF16X3><<<grid, 256, tc::Fmt<TC_BF16X3>::kBytes, s>>>(a, j0, nb, selftest);
    else if (form == TC_BF16X2)
        k_col_tc<TC_BF16X2><<<grid, 256, tc::Fmt<TC_BF16X2>::kBytes, s>>>(a, j0, nb, selftest);
    else
        k_col_tc<TC_TF32X2><<<grid, 256, tc::Fmt<TC_TF32X2>::kBytes, s>>>(a, j0, nb, selftest);
}
template <int F>
static cudaError_t set_attrs_tc_f() {
    cudaError_t e =
        cudaFuncSetAttribute(k_col_tc<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::Fmt<F>::kBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_col_tc<F>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}
template <int F>
static cudaError_t set_attrs_tc512_f() {
    return cudaFuncSetAttribute(k_col_tc512<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc::Fmt512<F>::kBytes);
}
cudaError_t set_attrs_tc() {
    cudaError_t e = set_attrs_tc_f<TC_TF32X2>();
    if (e == cudaSuccess) e = set_attrs_tc_f<TC_BF16X3>();
    if (e == cudaSuccess) e = set_attrs_tc_f<TC_BF16X2>();
    if (e == cudaSuccess) e = set_attrs_tc512_f<TC_TF32X2>();
    if (e == cudaSuccess) e = set_attrs_tc512_f<TC_BF16X3>();
    if (e == cudaSuccess) e = set_attrs_tc512_f<TC_BF16X2>();
    return e;
}

}  // namespace ptx
