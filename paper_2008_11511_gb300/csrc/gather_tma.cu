// Object numerator and denominator gathered per 32-column object tile (32, 16
// or 8 rows), fed by 3D tensor copies.  For each (frame j, mode k) meeting the
// tile, the window of Psi'_jk and of P_k under the tile is one box of the
// tile's rows x 34 columns
// (two extra columns so that the box starts on a 16-byte boundary) copied by
// the tensor memory accelerator into a ring of shared-memory stages; the parts
// of the window outside the frame arrive as zeros and add nothing.  One
// producer warp issues the copies, eight consumer warps accumulate
//   N_O(r) += conj(P_k(r - r_j)) Psi'_jk(r - r_j),  D_O(r) += |P_k(r - r_j)|^2
// in ascending j (the same order as the plain gather), one pixel column per
// lane, and write the tile once.
#include <cuda.h>

#include "kernels.cuh"

namespace ptx {

namespace {

constexpr int kT = 32;             // tile width (kObjTileW == 32)
constexpr int kBoxW = kT + 2;      // 34 columns: 272 bytes per box row
constexpr int kStages = 4;
constexpr int kConsumers = 8;      // warps
// one box: kRows rows of the tile (32, 16 or 8)
template <int kRows>
__host__ __device__ constexpr size_t box_bytes() { return sizeof(float2) * kBoxW * kRows; }

__device__ __forceinline__ uint32_t s_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
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
// bounded: gives up after ~2^31 clocks (about a second)
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!bar_try(bar, parity))
        if (clock64() - t0 > (1ll << 31)) return false;
    return true;
}
__device__ __forceinline__ void load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void flag_error(int* flag) {
    if (flag) {
        *(volatile int*)flag = 1;
        __threadfence_system();
    }
}

// Box origin of frame position p for the tile whose first row is y0 and whose
// column index is tx: column rounded down to even.
__device__ __forceinline__ void box_origin(int2 p, int y0, int tx, int& xs, int& ys, int& off) {
    const int xr = tx * kT - p.y;
    off = xr & 1;
    xs = xr - off;
    ys = y0 - p.x;
}

}  // namespace

template <int kRows>
__global__ void __launch_bounds__(32 * (kConsumers + 1), 2)
    k_obj_gather_t(const __grid_constant__ CUtensorMap tm_psi, const __grid_constant__ CUtensorMap tm_probe, ProbArgs a,
                   TileLists tl, int fuse_max) {
    constexpr size_t kBox = box_bytes<kRows>();
    constexpr uint32_t kTx = 2 * (uint32_t)kBox;
    constexpr int kQ = kRows / kConsumers;  // rows per consumer warp
    extern __shared__ __align__(128) unsigned char gsm[];
    float2(*st)[2][kRows * kBoxW] = reinterpret_cast<float2(*)[2][kRows * kBoxW]>(gsm);
    uint64_t* full = reinterpret_cast<uint64_t*>(gsm + kStages * 2 * kBox);
    uint64_t* empty = full + kStages;
    // column offset (0 or 1) of each stage's window, written by the producer
    // before its arrival on the stage's full barrier
    __shared__ int stage_off[kStages];
    const int t = blockIdx.x;
    const int tid = tl.tile_ids[t];
    const int ty = tid / tl.ntx, tx = tid - ty * tl.ntx;
    const int K = a.K;
    const int f0 = tl.tile_ptr[t], f1 = tl.tile_ptr[t + 1];
    const int nitems = (f1 - f0) * K;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            bar_init(s_u32(&full[s]), 1);
            bar_init(s_u32(&empty[s]), kConsumers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kConsumers) {  // producer warp
        // the tile's frames and their positions are staged in shared memory by
        // the whole warp, a chunk at a time, so that lane 0 issues the copies
        // without dependent global loads between them
        constexpr int kChunk = 128;
        __shared__ int pf_j[kChunk];
        __shared__ int2 pf_pos[kChunk];
        int ok = 1;
        int it = 0;
        const int nf = f1 - f0;
        for (int c0 = 0; c0 < nf && ok; c0 += kChunk) {
            const int cn = min(kChunk, nf - c0);
            __syncwarp();  // lane 0 is done with the previous chunk
            for (int q = lane; q < cn; q += 32) {
                const int j = tl.tile_frames[f0 + c0 + q];
                pf_j[q] = j;
                pf_pos[q] = a.pos[j];
            }
            __syncwarp();
            if (lane == 0) {
                for (int q = 0; q < cn && ok; ++q)
                    for (int k = 0; k < K; ++k, ++it) {
                        const int s = it % kStages;
                        if (it >= kStages) ok = bar_wait(s_u32(&empty[s]), ((it / kStages) - 1) & 1);
                        if (!ok) break;
                        const int j = pf_j[q];
                        int xs, ys, off;
                        box_origin(pf_pos[q], ty * kRows, tx, xs, ys, off);
                        stage_off[s] = off;
                        const uint32_t bar = s_u32(&full[s]);
                        bar_expect_tx(bar, kTx);
                        load_3d(s_u32(st[s][0]), &tm_psi, xs, ys, j * K + k, bar);
                        load_3d(s_u32(st[s][1]), &tm_probe, xs, ys, k, bar);
                    }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            it = __shfl_sync(0xffffffffu, it, 0);
        }
        if (lane == 0 && !ok) {
            flag_error(a.err_flag);
            // the copies already issued land before the block may exit
            for (int q = (it > kStages ? it - kStages : 0); q < it; ++q)
                bar_wait(s_u32(&full[q % kStages]), (q / kStages) & 1);
        }
        return;
    }

    // consumers: lane = tile column, rows warp + 8 q
    float2 n[kQ];
    float d[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        n[q] = make_float2(0.f, 0.f);
        d[q] = 0.f;
    }
    bool ok = true;
    for (int it = 0; it < nitems; ++it) {
        const int s = it % kStages;
        if (!bar_wait(s_u32(&full[s]), (it / kStages) & 1)) {
            ok = false;
            break;
        }
        const int off = stage_off[s];
        const float2* ps = st[s][0] + off + lane;
        const float2* pr = st[s][1] + off + lane;
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const int r = (warp + 8 * q) * kBoxW;
            const float2 pv = pr[r], sv = ps[r];
            const float2 c = cconjmul(pv, sv);
            n[q].x += c.x;
            n[q].y += c.y;
            d[q] = fmaf(pv.x, pv.x, fmaf(pv.y, pv.y, d[q]));
        }
        __syncwarp();
        if (lane == 0) bar_arrive(s_u32(&empty[s]));
    }
    if (!ok) flag_error(a.err_flag);
    const int x = tx * kT + lane;
    float dmax = 0.f;
    if (x < a.Wo) {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const int y = ty * kRows + warp + 8 * q;
            if (y < a.Ho) {
                a.acc_obj[(size_t)y * a.Wo + x] = make_float4(n[q].x, n[q].y, d[q], 0.f);
                dmax = fmaxf(dmax, d[q]);
            }
        }
    }
    if (fuse_max) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_down_sync(0xffffffffu, dmax, o));
        if (lane == 0 && dmax > 0.f) atomicMax(&a.maxbits[0], __float_as_uint(dmax));
    }
}

template <int kRows>
constexpr size_t gather_smem() { return kStages * 2 * box_bytes<kRows>() + 2 * kStages * sizeof(uint64_t); }

cudaError_t set_attrs_gather_tma() {
    cudaError_t e = cudaFuncSetAttribute(k_obj_gather_t<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gather_smem<32>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_obj_gather_t<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gather_smem<16>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_obj_gather_t<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gather_smem<8>());
    return e;
}

// tl.th selects the instantiation; the tensor maps' boxes are 34 x tl.th
void launch_obj_gather_tma(const void* tm_psi, const void* tm_probe, const ProbArgs& a, const TileLists& tl,
                           int ntiles, int fuse_max, cudaStream_t s) {
    const CUtensorMap& mp = *(const CUtensorMap*)tm_psi;
    const CUtensorMap& mq = *(const CUtensorMap*)tm_probe;
    constexpr int kTh = 32 * (kConsumers + 1);
    if (tl.th == 8)
        k_obj_gather_t<8><<<ntiles, kTh, gather_smem<8>(), s>>>(mp, mq, a, tl, fuse_max);
    else if (tl.th == 16)
        k_obj_gather_t<16><<<ntiles, kTh, gather_smem<16>(), s>>>(mp, mq, a, tl, fuse_max);
    else
        k_obj_gather_t<32><<<ntiles, kTh, gather_smem<32>(), s>>>(mp, mq, a, tl, fuse_max);
}

}  // namespace ptx
