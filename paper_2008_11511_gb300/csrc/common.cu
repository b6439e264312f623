// Normalisation, denominator maxima and FP64 log-likelihood reductions
// (second half of Psi2ObjProbe and the LLK operator's final sum).
#include "kernels.cuh"

namespace ptx {

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// max D_O and max D_P over the accumulators (both >= 0, so their bit patterns
// order like unsigned integers).
// Object numerator and denominator gathered per object tile from the stored
// exit waves and the (already updated) probe:
//   N_O(r) = sum_j sum_k conj(P_k(r - r_j)) Psi'_jk(r - r_j),  D_O(r) = sum_j sum_k |P_k(r - r_j)|^2
// over the frames whose patch contains r, in ascending j.  Each pixel is
// owned by one thread, so the accumulator is written without atomics.
__global__ void __launch_bounds__(256) k_obj_gather(ProbArgs a, TileLists tl, int fuse_max) {
    constexpr int TW = kObjTileW, TH = kObjTileH;
    constexpr int RS = 256 / TW;          // rows covered by the block's threads at once
    constexpr int Q = TW * TH / 256;      // pixels per thread (at most): rows wy + RS q of column x
    const int Qr = TW * tl.th / 256;      // this tile height's
    const int t = blockIdx.x;
    const int tid = tl.tile_ids[t];
    const int ty = tid / tl.ntx, tx = tid - ty * tl.ntx;
    const int wy = threadIdx.x / TW;
    const int x = tx * TW + threadIdx.x % TW;
    const int N = a.N, K = a.K;
    float2 n[Q];
    float d[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        n[q] = make_float2(0.f, 0.f);
        d[q] = 0.f;
    }
    const int f0 = tl.tile_ptr[t], f1 = tl.tile_ptr[t + 1];
    const int y0 = ty * tl.th + wy;
    // F frames per step: all their loads are issued before any is used, so each
    // thread keeps up to 2 F Q loads in flight (the loop is latency-bound otherwise)
    constexpr int F = 4;
    for (int f = f0; f < f1; f += F) {
        float2 pr[F][Q], ps[F][Q];
        bool ok[F][Q];
        for (int k = 0; k < K; ++k) {
#pragma unroll
            for (int u = 0; u < F; ++u) {
                const int fi = f + u;
                const int j = fi < f1 ? tl.tile_frames[fi] : 0;
                const int2 p = a.pos[j];
                const int px = x - p.y;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int py = y0 + RS * q - p.x;
                    ok[u][q] = q < Qr && fi < f1 && px >= 0 && px < N && py >= 0 && py < N;
                    const size_t off = ok[u][q] ? ((size_t)k * N + py) * N + px : 0;
                    pr[u][q] = ok[u][q] ? __ldg(a.probe + off) : make_float2(0.f, 0.f);
                    ps[u][q] = ok[u][q] ? __ldcs(a.psi + (size_t)j * K * N * N + off) : make_float2(0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < F; ++u)
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const float2 c = cconjmul(pr[u][q], ps[u][q]);
                    n[q].x += c.x;
                    n[q].y += c.y;
                    d[q] = fmaf(pr[u][q].x, pr[u][q].x, fmaf(pr[u][q].y, pr[u][q].y, d[q]));
                }
        }
    }
    float dmax = 0.f;
    if (x < a.Wo) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int y = y0 + RS * q;
            if (q < Qr && y < a.Ho) {
                a.acc_obj[(size_t)y * a.Wo + x] = make_float4(n[q].x, n[q].y, d[q], 0.f);
                dmax = fmaxf(dmax, d[q]);
            }
        }
    }
    // max D_O for the inertia term, when the normalisation follows directly
    // (D_O >= 0, so float bits order like unsigned integers; tiles met by no
    // frame keep D_O = 0)
    if (fuse_max) {
        dmax = warp_max(dmax);
        if ((threadIdx.x & 31) == 0 && dmax > 0.f) atomicMax(&a.maxbits[0], __float_as_uint(dmax));
    }
}

__global__ void k_den_max(ProbArgs a, int upd_obj, int upd_probe) {
    float mo = 0.f, mp = 0.f;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (upd_obj) {
        const size_t n = (size_t)a.Ho * a.Wo;
        for (size_t i = i0; i < n; i += stride) mo = fmaxf(mo, a.acc_obj[i].z);
    }
    if (upd_probe) {
        const size_t n = (size_t)a.N * a.N;
        for (size_t i = i0; i < n; i += stride) mp = fmaxf(mp, a.acc_probe[i].z);
    }
    mo = warp_max(mo);
    mp = warp_max(mp);
    if ((threadIdx.x & 31) == 0) {
        if (mo > 0.f) atomicMax(&a.maxbits[0], __float_as_uint(mo));
        if (mp > 0.f) atomicMax(&a.maxbits[1], __float_as_uint(mp));
    }
}

// O <- (N_O + d_O O) / (D_O + d_O), d_O = alpha_obj max D_O (unchanged where the
// denominator is 0); the same for each probe mode with D_P; accumulators cleared.
__global__ void k_normalise(ProbArgs a, float alpha_obj, float alpha_probe, int upd_obj, int upd_probe) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (upd_obj) {
        const float d = alpha_obj * __uint_as_float(a.maxbits[0]);
        const size_t n = (size_t)a.Ho * a.Wo;
        for (size_t i = i0; i < n; i += stride) {
            const float4 v = a.acc_obj[i];
            const float den = v.z + d;
            if (den > 0.f) {
                const float2 o = a.obj[i];
                a.obj[i] = make_float2((v.x + d * o.x) / den, (v.y + d * o.y) / den);
            }
            a.acc_obj[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    if (upd_probe) {
        const float d = alpha_probe * __uint_as_float(a.maxbits[1]);
        const size_t n = (size_t)a.K * a.N * a.N;
        for (size_t i = i0; i < n; i += stride) {
            const float4 v = a.acc_probe[i];
            const float den = v.z + d;
            if (den > 0.f) {
                const float2 o = a.probe[i];
                a.probe[i] = make_float2((v.x + d * o.x) / den, (v.y + d * o.y) / den);
            }
            a.acc_probe[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

__device__ double block_reduce_llk(const double* part, size_t n) {
    __shared__ double red[32];
    double s = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;
}

__global__ void k_llk_reduce(ProbArgs a, int nparts_per_frame, double* out) {
    double r = block_reduce_llk(a.llk_part, (size_t)a.J * nparts_per_frame);
    if (threadIdx.x == 0) *out = r;
}

// The cycle's LLK: block b sums the contiguous chunk b of the partial sums
// into ctl->l2[b]; the last block to finish sums l2[0 .. gridDim.x) in index
// order, so the result does not depend on the blocks' timing.
__global__ void k_cycle_end(Ctl* ctl, ProbArgs a, int p, int nparts_per_frame, int last_problem) {
    __shared__ bool is_last;
    const size_t n = (size_t)a.J * nparts_per_frame;
    const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const size_t b0 = (size_t)blockIdx.x * chunk;
    const size_t nb = b0 < n ? (n - b0 < chunk ? n - b0 : chunk) : 0;
    const double s = block_reduce_llk(a.llk_part + b0, nb);
    if (threadIdx.x == 0) {
        ctl->l2[blockIdx.x] = s;
        __threadfence();
        is_last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const double r = block_reduce_llk(ctl->l2, gridDim.x);
    if (threadIdx.x == 0) {
        if (ctl->llk_out) ctl->llk_out[(size_t)ctl->cycle * ctl->nprob + p] = r;
        a.maxbits[0] = 0u;
        a.maxbits[1] = 0u;
        ctl->ticket = 0u;
        if (last_problem) ctl->cycle += 1;
    }
}

// Background update of an AP cycle: B <- B * (1/J) sum_j I_o / (I_c + B) on
// unmasked pixels, then the sums are cleared for the next cycle.
__global__ void k_bg_update(float* bg, float* acc, const uint8_t* mask, int n, float inv_j) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!mask[i]) bg[i] *= acc[i] * inv_j;
        acc[i] = 0.f;
    }
}

// Self-test of the bounded-wait failure path: one thread waits for a
// shared-memory flag that nothing sets, at most limit_ns of the global timer
// (and at most 2^31 SM clocks), then records the give-up in err_flag as the
// tensor-copy waits do.  The wait always ends.
__global__ void k_wait_selftest(int* err_flag, unsigned long long limit_ns) {
    __shared__ volatile int never;
    never = 0;
    __syncthreads();
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    const long long c0 = clock64();
    while (!never) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns || clock64() - c0 > (1ll << 31)) {
            if (err_flag) {
                *(volatile int*)err_flag = 1;
                __threadfence_system();
            }
            return;
        }
    }
}

// FP32 FMA throughput probe: every thread runs `iters` rounds of 16 independent
// FMA chains (32 flop per round), enough independent work per warp to keep the
// FMA pipes issuing every cycle.  The chains' sum goes to sink[thread] so that
// nothing is dropped by the compiler; a, b keep the values bounded.
__global__ void __launch_bounds__(256) k_fma_peak(float* __restrict__ sink, int iters, float a, float b) {
    float x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = fmaf(x[i], a, b);
    }
    float t = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) t += x[i];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// Photon counts (uint16) to the float32 intensities the passes read: 8 counts
// (16 bytes) per thread and step, exact (every uint16 is a float32 integer).
__global__ void k_counts_to_float(const uint16_t* __restrict__ src, float* __restrict__ dst, size_t n) {
    const size_t n8 = n / 8;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += stride) {
        const uint4 v = __ldcs(reinterpret_cast<const uint4*>(src) + i);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        float4 lo, hi;
        lo.x = (float)(w[0] & 0xffffu); lo.y = (float)(w[0] >> 16);
        lo.z = (float)(w[1] & 0xffffu); lo.w = (float)(w[1] >> 16);
        hi.x = (float)(w[2] & 0xffffu); hi.y = (float)(w[2] >> 16);
        hi.z = (float)(w[3] & 0xffffu); hi.w = (float)(w[3] >> 16);
        float4* d = reinterpret_cast<float4*>(dst) + 2 * i;
        __stcs(d, lo);  // streaming stores: the intensities are read a cycle later,
        __stcs(d + 1, hi);  // they should not push the work stack out of L2
    }
    // the tail (n not a multiple of 8)
    for (size_t i = 8 * n8 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = (float)src[i];
}

// One-byte counts to float32: 16 counts (16 bytes) per thread and step.
__global__ void k_counts8_to_float(const uint8_t* __restrict__ src, float* __restrict__ dst, size_t n) {
    const size_t n16 = n / 16;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
        const uint4 v = __ldcs(reinterpret_cast<const uint4*>(src) + i);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        float4* d = reinterpret_cast<float4*>(dst) + 4 * i;
#pragma unroll
        for (int q = 0; q < 4; ++q)  // streaming stores, as in k_counts_to_float
            __stcs(d + q, make_float4((float)(w[q] & 0xffu), (float)((w[q] >> 8) & 0xffu),
                                      (float)((w[q] >> 16) & 0xffu), (float)(w[q] >> 24)));
    }
    // the tail (n not a multiple of 16)
    for (size_t i = 16 * n16 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = (float)src[i];
}

// The escapes of the one-byte form: dst[index[k]] = value[k] for the indices
// inside the n elements of dst (others are skipped).
__global__ void k_counts8_escapes(const uint32_t* __restrict__ index, const uint16_t* __restrict__ value,
                                  float* __restrict__ dst, size_t n_esc, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_esc; k += stride) {
        const uint32_t i = index[k];
        if (i < n) dst[i] = (float)value[k];
    }
}

__global__ void k_set_ctl(Ctl* ctl, double* llk_out, int nprob) {
    ctl->llk_out = llk_out;
    ctl->cycle = 0;
    ctl->ticket = 0u;
    ctl->nprob = nprob;
    ctl->err = 0;
}

}  // namespace ptx

namespace ptx {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// <G,G>, <G,Gp>, <Gp,Gp> over the object and probe parts: FP64 sums per block
// into cg_part[block][0..2] (k_cg_reduce adds the blocks in index order, so the
// result does not depend on scheduling).  kCgBlocks blocks of 256 threads.
__global__ void k_cg_dots(CgArgs c) {
    double gg = 0.0, ggp = 0.0, gpgp = 0.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t tot = c.n_obj + c.n_probe;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += stride) {
        const bool o = i < c.n_obj;
        const size_t k = o ? i : i - c.n_obj;
        const float2 g = o ? c.g_obj[k] : c.g_probe[k];
        const float2 q = o ? c.gp_obj[k] : c.gp_probe[k];
        gg += (double)g.x * g.x + (double)g.y * g.y;
        ggp += (double)g.x * q.x + (double)g.y * q.y;
        gpgp += (double)q.x * q.x + (double)q.y * q.y;
    }
    __shared__ double red_s[256 / 32];
    const double t0 = block_sum_double<256>(gg, red_s);
    __syncthreads();
    const double t1 = block_sum_double<256>(ggp, red_s);
    __syncthreads();
    const double t2 = block_sum_double<256>(gpgp, red_s);
    if (threadIdx.x == 0) {
        c.cg_part[3 * blockIdx.x + 0] = t0;
        c.cg_part[3 * blockIdx.x + 1] = t1;
        c.cg_part[3 * blockIdx.x + 2] = t2;
    }
}

// cg[0..2] = sums of the kCgBlocks partials of k_cg_dots, in a fixed order.
// One block of 256 threads.
__global__ void k_cg_reduce(CgArgs c) {
    __shared__ double red_s[256 / 32];
    for (int q = 0; q < 3; ++q) {
        double v = 0.0;
        for (int b = threadIdx.x; b < kCgBlocks; b += 256) v += c.cg_part[3 * b + q];
        const double t = block_sum_double<256>(v, red_s);
        if (threadIdx.x == 0) c.cg[q] = t;
        __syncthreads();
    }
}

// Polak-Ribiere: beta = max(0, (<G,G> - <G,Gp>) / <Gp,Gp>) (0 without a previous
// gradient); D <- -G + beta D; Gp <- G.
__global__ void k_cg_direction(CgArgs c) {
    const double den = c.cg[2];
    const double beta = den > 0.0 ? fmax(0.0, (c.cg[0] - c.cg[1]) / den) : 0.0;
    const float b = (float)beta;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t tot = c.n_obj + c.n_probe;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += stride) {
        const bool o = i < c.n_obj;
        const size_t k = o ? i : i - c.n_obj;
        float2* g = o ? c.g_obj + k : c.g_probe + k;
        float2* gp = o ? c.gp_obj + k : c.gp_probe + k;
        float2* d = o ? c.d_obj + k : c.d_probe + k;
        const float2 gv = *g;
        const float2 dv = *d;
        *d = make_float2(fmaf(b, dv.x, -gv.x), fmaf(b, dv.y, -gv.y));
        *gp = gv;
    }
}

// alpha = -L'(0) / L''(0) (0 when L''(0) <= 0); O += alpha D_O, P += alpha D_P.
__global__ void k_cg_step(CgArgs c, float2* obj, float2* probe) {
    const double l1 = c.cg[3], l2 = c.cg[4];
    const float alpha = l2 > 0.0 ? (float)(-l1 / l2) : 0.f;
    if (blockIdx.x == 0 && threadIdx.x == 0) c.cg[5] = l2 > 0.0 ? -l1 / l2 : 0.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t tot = c.n_obj + c.n_probe;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += stride) {
        const bool o = i < c.n_obj;
        const size_t k = o ? i : i - c.n_obj;
        float2* z = o ? obj + k : probe + k;
        const float2 d = o ? c.d_obj[k] : c.d_probe[k];
        const float2 v = *z;
        *z = make_float2(fmaf(alpha, d.x, v.x), fmaf(alpha, d.y, v.y));
    }
}

// Sum of the line-search partials (pairs) in a fixed order: out[0] = L'(0), out[1] = L''(0).
__global__ void k_ls_reduce(const double* part, size_t nparts, double* out) {
    __shared__ double red[2][32];
    double a = 0.0, b = 0.0;
    for (size_t i = threadIdx.x; i < nparts; i += blockDim.x) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a;
        red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        a = threadIdx.x < (blockDim.x >> 5) ? red[0][threadIdx.x] : 0.0;
        b = threadIdx.x < (blockDim.x >> 5) ? red[1][threadIdx.x] : 0.0;
        a = warp_sum_d(a);
        b = warp_sum_d(b);
        if (threadIdx.x == 0) {
            out[0] = a;
            out[1] = b;
        }
    }
}

}  // namespace ptx
