// Forward and backward row passes of the cycle with the DFT stages of each
// row transform on the tensor cores (the split-precision form of the paper's
// FT / IFT operators on the rows): 256^2 frames with one probe mode (two
// 16-point stages) and 512^2 frames with any number of modes (a 16-point and a
// 32-point stage, at the end of this file).  Same inputs, outputs and
// work-stack layout as the register row passes, so either can run beside the
// FP32 or the tensor-core column pass.
//
// At 256^2 a block holds a band of 16 rows as two independent halves of 8 rows
// (tc::Pipe256: own A tile, mbarrier, TMEM columns and named barrier).  Thread
// u of half h is (row 8 h + u / 16 of the band, index q = u % 16) and owns row
// u of its half's tile in every stage; the stage-2 vectors of a row are the 16
// tile rows of that row (16 (u / 16) + k).  A block loops over frames (the
// matrices, twiddles and TMEM set up once).
#include <algorithm>

#include "tc.cuh"

namespace ptx {

// grid (16 bands, frame slots), 256 threads.  X = P O (AP, and the
// initialising DM cycle) or 2 P O - Psi (DM) along row y of each frame, its
// 256-point row DFT written to the work stack (unnormalised, as the FP32 pass).
template <int F, bool kDM>
__global__ void __launch_bounds__(256, 2) k_row_fwd_tc(ProbArgs a, int j0, int nb) {
    using namespace tc;
    extern __shared__ unsigned char smraw[];
    const int t = threadIdx.x, h = t >> 7, u = t & 127, cl = u >> 4, q = u & 15;
    const int y = blockIdx.x * 16 + 8 * h + cl;
    Pipe256<F> pp;
    pp.setup(smraw, false);
    const float2* tw = pp.tw;
    const float2* pr = a.probe + (size_t)y * N + q;  // probe row y, columns q + 16 n2
    float2 v[16];
    float o[32];
    bool good = true, bad = false;
    for (int b = blockIdx.y; b < nb; b += gridDim.y) {
        const int j = j0 + b;
        const int2 p = a.pos[j];
        // stage-1 vector (row y, n1 = q): X[q + 16 n2], n2 = 0..15
        const float2* ob = a.obj + (size_t)(p.x + y) * a.Wo + p.y + q;
        if constexpr (kDM) {
            const float2* ps = a.psi + ((size_t)j * N + y) * N + q;
            const uint64_t ef = policy_evict_first();
#pragma unroll
            for (int n2 = 0; n2 < 16; ++n2) v[n2] = ld_hint(ps + 16 * n2, ef);
#pragma unroll
            for (int n2 = 0; n2 < 16; ++n2) {
                const float2 phi = cmul(__ldg(pr + 16 * n2), ob[16 * n2]);
                v[n2] = make_float2(2.f * phi.x - v[n2].x, 2.f * phi.y - v[n2].y);
            }
        } else {
#pragma unroll
            for (int n2 = 0; n2 < 16; ++n2) v[n2] = cmul(__ldg(pr + 16 * n2), ob[16 * n2]);
        }
        pp.put_row(v);
        good = pp.stage(0, o);
        if (good) {
            // twiddle w^(n1 k2) and the transpose into the vectors (row, k2): tile rows 16 cl + k2
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) {
                const float2 yv = make_float2(o[2 * k2], o[2 * k2 + 1]);
                v[k2] = k2 == 0 ? yv : cmul(yv, tw_get<N, -1>(tw, k2, q));
            }
            pp.template put_col<1>(v, 16 * cl, q);
            good = pp.stage(0, o);
        }
        if (good) {
            // X^[k2 + 16 k1] of row y (thread = vector (row, k2 = q))
            float2* dst = a.spec + ((size_t)b * N + y) * N + q;
            const uint64_t el = policy_evict_last();
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) st_hint(dst + 16 * k1, make_float2(o[2 * k1], o[2 * k1 + 1]), el);
        }
        bad = __syncthreads_or(!good);
        if (bad) break;
    }
    pp.finish(good, bad, a.err_flag);
}

// grid (16 bands, G frame slots), 256 threads.  The inverse row DFT of the
// work stack's row y gives the correction D; Psi' = P O + D is stored (AP and
// DM alike), and with upd_probe the probe numerator conj(O) Psi' and
// denominator |O|^2 of the thread's 16 pixels are summed in registers over the
// block's frames (slot, slot + G, ...) and added to the accumulator once.
template <int F>
__global__ void __launch_bounds__(256, 2) k_row_bwd_tc(ProbArgs a, int j0, int nb, int upd_probe) {
    using namespace tc;
    extern __shared__ unsigned char smraw[];
    const int t = threadIdx.x, h = t >> 7, u = t & 127, cl = u >> 4, q = u & 15;
    const int y = blockIdx.x * 16 + 8 * h + cl;
    Pipe256<F> pp;
    pp.setup(smraw, false);
    const float2* tw = pp.tw;
    const float2* pr = a.probe + (size_t)y * N + q;  // probe row y, columns q + 16 k1
    float2 np[16];
    float dp[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        np[k] = make_float2(0.f, 0.f);
        dp[k] = 0.f;
    }
    float2 v[16];
    float o[32];
    bool good = true, bad = false;
    for (int b = blockIdx.y; b < nb; b += gridDim.y) {
        const int j = j0 + b;
        const int2 p = a.pos[j];
        // stage-1 vector (row y, k2 = q): the work stack's D^[q + 16 k1], its last read
        {
            const float2* src = a.spec + ((size_t)b * N + y) * N + q;
            const uint64_t ef = policy_evict_first();
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) v[k1] = ld_hint(src + 16 * k1, ef);
        }
        pp.put_row(v);
        good = pp.stage(1, o);
        if (good) {
            // twiddle w^(+k2 kk) and the transpose into the vectors (row, kk): tile rows 16 cl + kk
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const float2 yv = make_float2(o[2 * kk], o[2 * kk + 1]);
                v[kk] = kk == 0 ? yv : cmul(yv, tw_get<N, +1>(tw, q, kk));
            }
            pp.template put_col<1>(v, 16 * cl, q);
            good = pp.stage(1, o);
        }
        if (good) {
            // D at the pixels kk + 16 k1' of row y (thread = vector (row, kk = q))
            const float2* ob = a.obj + (size_t)(p.x + y) * a.Wo + p.y + q;
            float2* ps = a.psi + ((size_t)j * N + y) * N + q;
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                const float2 obv = ob[16 * k1];
                const float2 wv = cadd(cmul(__ldg(pr + 16 * k1), obv), make_float2(o[2 * k1], o[2 * k1 + 1]));
                __stcs(ps + 16 * k1, wv);
                if (upd_probe) {
                    const float2 tt = cconjmul(obv, wv);
                    np[k1].x += tt.x;
                    np[k1].y += tt.y;
                    dp[k1] += cnorm(obv);
                }
            }
        }
        bad = __syncthreads_or(!good);
        if (bad) break;
    }
    if (upd_probe && !bad) {
        float4* acc = a.acc_probe + (size_t)y * N + q;
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) red_add_v4(acc + 16 * k1, np[k1].x, np[k1].y, dp[k1], 0.f);
    }
    pp.finish(good, bad, a.err_flag);
}

// ---------------------------------------------------------------------------
// The 512-point row transforms (512 = 16 x 32, tc::Pipe512), any number of
// probe modes (the row passes treat the modes independently).  A 512-thread
// block holds a band of 16 rows: thread t owns the stage-A vector (row t / 32,
// n1 = t % 32) and, in stage B, half h = t / 256 of the vector (row r / 16,
// k2 = r % 16), r = t % 256, so that the loads and stores along a row are
// contiguous over the threads.
// ---------------------------------------------------------------------------

// grid (32 bands, frame-mode slots), 512 threads.  Same outputs as the FP32
// forward row pass at 512^2.
template <int F, bool kDM>
__global__ void __launch_bounds__(512, 1) k_row_fwd_tc512(ProbArgs a, int j0, int nb) {
    using namespace tc;
    constexpr int N = 512;
    extern __shared__ unsigned char smraw[];
    const int t = threadIdx.x, K = a.K;
    const int lineA = t >> 5, n1 = t & 31;                             // stage-A vector
    const int r2 = t & 255, h = t >> 8, lineB = r2 >> 4, k2 = r2 & 15;  // stage-B row and half
    const int yA = blockIdx.x * 16 + lineA, yB = blockIdx.x * 16 + lineB;
    Pipe512<F> pp;
    pp.setup(smraw);
    const float2* tw = pp.tw;
    float2 v[16];
    float o[32];
    bool good = true;
    for (int it = blockIdx.y; it < nb * K; it += gridDim.y) {
        const int b = it / K, k = it - b * K, j = j0 + b;
        const int2 p = a.pos[j];
        // stage-A vector (row yA, n1): X[n1 + 32 n2], n2 = 0..15
        const float2* pr = a.probe + ((size_t)k * N + yA) * N + n1;
        const float2* ob = a.obj + (size_t)(p.x + yA) * a.Wo + p.y + n1;
        if constexpr (kDM) {
            const float2* ps = a.psi + (((size_t)j * K + k) * N + yA) * N + n1;
            const uint64_t ef = policy_evict_first();
#pragma unroll
            for (int n2 = 0; n2 < 16; ++n2) v[n2] = ld_hint(ps + 32 * n2, ef);
#pragma unroll
            for (int n2 = 0; n2 < 16; ++n2) {
                const float2 phi = cmul(__ldg(pr + 32 * n2), ob[32 * n2]);
                v[n2] = make_float2(2.f * phi.x - v[n2].x, 2.f * phi.y - v[n2].y);
            }
        } else {
#pragma unroll
            for (int n2 = 0; n2 < 16; ++n2) v[n2] = cmul(__ldg(pr + 32 * n2), ob[32 * n2]);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) pp.put(0, t, i, v[i]);
        good = pp.stage(false, 0, o);
        if (good) {
            // twiddle w^(n1 kk) and the transpose into the stage-B rows (row, kk): 16 lineA + kk
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const float2 yv = make_float2(o[2 * kk], o[2 * kk + 1]);
                pp.put(n1 >> 4, 16 * lineA + kk, n1 & 15, kk == 0 ? yv : cmul(yv, tw_get<N, -1>(tw, kk, n1)));
            }
            good = pp.stage(true, 0, o);
        }
        if (good) {
            // X^[k2 + 16 k1] of row yB, k1 = 16 h + i
            float2* dst = a.spec + (((size_t)b * K + k) * N + yB) * N + k2 + 256 * h;
            const uint64_t el = policy_evict_last();
#pragma unroll
            for (int i = 0; i < 16; ++i) st_hint(dst + 16 * i, make_float2(o[2 * i], o[2 * i + 1]), el);
        }
        if (__syncthreads_or(!good)) {
            good = false;
            break;
        }
    }
    pp.finish(good, a.err_flag);
}

// grid (32 bands, G frame slots x K modes), 512 threads; blockIdx.y = slot K +
// mode.  The inverse row DFT of the work stack's rows gives D; Psi' = P_k O + D
// is stored and, with upd_probe, the probe sums of the thread's 16 pixels are
// kept in registers over the block's frames and added once.
template <int F>
__global__ void __launch_bounds__(512, 1) k_row_bwd_tc512(ProbArgs a, int j0, int nb, int upd_probe) {
    using namespace tc;
    constexpr int N = 512;
    extern __shared__ unsigned char smraw[];
    const int t = threadIdx.x, K = a.K;
    const int lineA = t >> 5, n1 = t & 31;
    const int r2 = t & 255, h = t >> 8, lineB = r2 >> 4, k2 = r2 & 15;
    const int yA = blockIdx.x * 16 + lineA, yB = blockIdx.x * 16 + lineB;
    const int slot = blockIdx.y / K, k = blockIdx.y - slot * K, G = gridDim.y / K;
    Pipe512<F> pp;
    pp.setup(smraw);
    const float2* tw = pp.tw;
    const float2* pr = a.probe + ((size_t)k * N + yA) * N + n1;  // probe row yA, columns n1 + 32 i
    float2 np[16];
    float dp[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        np[i] = make_float2(0.f, 0.f);
        dp[i] = 0.f;
    }
    float2 v[16];
    float o[32];
    bool good = true;
    for (int b = slot; b < nb; b += G) {
        const int j = j0 + b;
        const int2 p = a.pos[j];
        // stage-B vector (row yB, k2), half h: D^[k2 + 16 k1], k1 = 16 h + i (the stack's last read)
        {
            const float2* src = a.spec + (((size_t)b * K + k) * N + yB) * N + k2 + 256 * h;
            const uint64_t ef = policy_evict_first();
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = ld_hint(src + 16 * i, ef);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) pp.put(h, r2, i, v[i]);
        good = pp.stage(true, 1, o);
        if (good) {
            // twiddle w^(+k2 kk), kk = 16 h + i, and the transpose into the stage-A rows (row, kk): 32 lineB + kk
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int kk = 16 * h + i;
                const float2 yv = make_float2(o[2 * i], o[2 * i + 1]);
                pp.put(0, 32 * lineB + kk, k2, (k2 == 0 || kk == 0) ? yv : cmul(yv, tw_get<N, +1>(tw, k2, kk)));
            }
            good = pp.stage(false, 1, o);
        }
        if (good) {
            // D at the pixels n1 + 32 i of row yA (thread = stage-A row t = (row, kk = n1))
            const float2* ob = a.obj + (size_t)(p.x + yA) * a.Wo + p.y + n1;
            float2* ps = a.psi + (((size_t)j * K + k) * N + yA) * N + n1;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float2 obv = ob[32 * i];
                const float2 wv = cadd(cmul(__ldg(pr + 32 * i), obv), make_float2(o[2 * i], o[2 * i + 1]));
                __stcs(ps + 32 * i, wv);
                if (upd_probe) {
                    const float2 tt = cconjmul(obv, wv);
                    np[i].x += tt.x;
                    np[i].y += tt.y;
                    dp[i] += cnorm(obv);
                }
            }
        }
        if (__syncthreads_or(!good)) {
            good = false;
            break;
        }
    }
    if (upd_probe && good) {
        float4* acc = a.acc_probe + ((size_t)k * N + yA) * N + n1;
#pragma unroll
        for (int i = 0; i < 16; ++i) red_add_v4(acc + 32 * i, np[i].x, np[i].y, dp[i], 0.f);
    }
    pp.finish(good, a.err_flag);
}

// Frame slots of the tensor-core row passes: two blocks per SM over the 16
// bands; each block runs about nb / slots frames.
static int tc_row_slots(int nb) {
    const int slots = std::max(1, 2 * sm_count() / 16);
    const int per = (nb + slots - 1) / slots;
    return (nb + per - 1) / per;
}

template <int F>
static void launch_row_fwd_tc512_f(const ProbArgs& a, int j0, int nb, bool dm, cudaStream_t s) {
    // one block per SM over the 32 bands: each block runs about nb K / slots frame-modes
    const int items = nb * a.K;
    const int slots = std::max(1, sm_count() / 32);
    const int per = (items + slots - 1) / slots;
    dim3 grid(32, (items + per - 1) / per);
    if (dm)
        k_row_fwd_tc512<F, true><<<grid, 512, tc::Fmt512<F>::kBytes, s>>>(a, j0, nb);
    else
        k_row_fwd_tc512<F, false><<<grid, 512, tc::Fmt512<F>::kBytes, s>>>(a, j0, nb);
}

void launch_row_fwd_tc(const ProbArgs& a, int j0, int nb, bool dm, int form, cudaStream_t s) {
    if (a.N == 512) {
        if (form == TC_BF16X3)
            launch_row_fwd_tc512_f<TC_BF16X3>(a, j0, nb, dm, s);
        else if (form == TC_BF16X2)
            launch_row_fwd_tc512_f<TC_BF16X2>(a, j0, nb, dm, s);
        else
            launch_row_fwd_tc512_f<TC_TF32X2>(a, j0, nb, dm, s);
        return;
    }
    dim3 grid(16, tc_row_slots(nb));
    using namespace tc;
    if (form == TC_BF16X3) {
        if (dm)
            k_row_fwd_tc<TC_BF16X3, true><<<grid, 256, Fmt<TC_BF16X3>::kBytes, s>>>(a, j0, nb);
        else
            k_row_fwd_tc<TC_BF16X3, false><<<grid, 256, Fmt<TC_BF16X3>::kBytes, s>>>(a, j0, nb);
    } else if (form == TC_BF16X2) {
        if (dm)
            k_row_fwd_tc<TC_BF16X2, true><<<grid, 256, Fmt<TC_BF16X2>::kBytes, s>>>(a, j0, nb);
        else
            k_row_fwd_tc<TC_BF16X2, false><<<grid, 256, Fmt<TC_BF16X2>::kBytes, s>>>(a, j0, nb);
    } else {
        if (dm)
            k_row_fwd_tc<TC_TF32X2, true><<<grid, 256, Fmt<TC_TF32X2>::kBytes, s>>>(a, j0, nb);
        else
            k_row_fwd_tc<TC_TF32X2, false><<<grid, 256, Fmt<TC_TF32X2>::kBytes, s>>>(a, j0, nb);
    }
}

void launch_row_bwd_tc(const ProbArgs& a, int j0, int nb, int G, int upd_probe, int form, cudaStream_t s) {
    using namespace tc;
    if (a.N == 512) {
        // one block per SM over the 32 bands and the modes: frame slots per (band, mode)
        const int Gs = std::max(1, std::min(nb, sm_count() / (32 * a.K)));
        dim3 grid(32, Gs * a.K);
        if (form == TC_BF16X3)
            k_row_bwd_tc512<TC_BF16X3><<<grid, 512, Fmt512<TC_BF16X3>::kBytes, s>>>(a, j0, nb, upd_probe);
        else if (form == TC_BF16X2)
            k_row_bwd_tc512<TC_BF16X2><<<grid, 512, Fmt512<TC_BF16X2>::kBytes, s>>>(a, j0, nb, upd_probe);
        else
            k_row_bwd_tc512<TC_TF32X2><<<grid, 512, Fmt512<TC_TF32X2>::kBytes, s>>>(a, j0, nb, upd_probe);
        return;
    }
    dim3 grid(16, std::max(1, std::min(G, nb)));
    if (form == TC_BF16X3)
        k_row_bwd_tc<TC_BF16X3><<<grid, 256, Fmt<TC_BF16X3>::kBytes, s>>>(a, j0, nb, upd_probe);
    else if (form == TC_BF16X2)
        k_row_bwd_tc<TC_BF16X2><<<grid, 256, Fmt<TC_BF16X2>::kBytes, s>>>(a, j0, nb, upd_probe);
    else
        k_row_bwd_tc<TC_TF32X2><<<grid, 256, Fmt<TC_TF32X2>::kBytes, s>>>(a, j0, nb, upd_probe);
}

template <int F>
static cudaError_t set_attrs_row_tc_f() {
    const int bytes = (int)tc::Fmt<F>::kBytes;
    cudaError_t e = cudaFuncSetAttribute(k_row_fwd_tc<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_row_fwd_tc<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_row_bwd_tc<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    const int b512 = (int)tc::Fmt512<F>::kBytes;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_row_fwd_tc512<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b512);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_row_fwd_tc512<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b512);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_row_bwd_tc512<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, b512);
    return e;
}
cudaError_t set_attrs_row_tc() {
    cudaError_t e = set_attrs_row_tc_f<TC_TF32X2>();
    if (e == cudaSuccess) e = set_attrs_row_tc_f<TC_BF16X3>();
    if (e == cudaSuccess) e = set_attrs_row_tc_f<TC_BF16X2>();
    return e;
}

}  // namespace ptx
