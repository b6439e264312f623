// Persistent schedule of the cycle's batch passes: the forward row pass, the
// column pass and the backward row pass of every batch of every problem of a
// handle run as work items of ONE launch (the stacks of frames of the paper's
// Section 4, for many scans at once; the overlap update of each problem runs
// after it, in the same CUDA graph).
//
// Work list.  The batches of all problems are numbered g = 0 .. nbatch - 1;
// batch g uses work-stack slot g mod kSlots.  The items are handed out in
// pipeline order, step s = 0 .. nbatch + 1: the row items of batch s, the
// column items of batch s - 1, the backward items of batch s - 2.  A forward
// row or column item covers kPersFrames frames of one band or column block.
// A block takes item indices from a global counter (the next one while the
// current item runs), finds the segment (batch, pass) by scanning forward from
// its last one, and waits until the items it depends on are done:
//   column items of g   after every forward row item of g,
//   backward items of g after every column item of g,
//   forward items of g  after every backward item of g - kSlots (the slot's
//                       previous batch has been read out).
// Each dependency is on items earlier in the list, which running blocks have
// taken and will finish: the lowest unfinished item's dependencies are all
// done, and its block is working on it (a block's other index, the one taken
// ahead, is higher), so the schedule cannot deadlock.  Every wait is bounded (about 2^31 SM
// clocks); a wait that runs out sets the abort flag, which every block checks
// before taking an item, and the handle's error flag, and the launch drains.
//
// The pass bodies are those of the standalone kernels (body_*.inc), included
// here with the block coordinates taken from the item; the sizes are the
// register-resident ones of the batched workloads (128, 192, 256, 384, 512),
// one probe mode, far field, no background.
#include "kernels.cuh"

namespace ptx {

namespace pers {

constexpr int kSlots = kPersSlots;

// Each (size, pass) body is compiled as a function of its own (not inlined
// into the dispatch), so that each keeps its own register allocation; the
// item's problem arguments live in shared memory.
template <int N, bool kDM>
__device__ __noinline__ void row_fwd(const ProbArgs& a, int j0, int pbx, int pby) {
#define PTX_BX pbx
#define PTX_BY pby
#include "body_row_fwd.inc"
#undef PTX_BX
#undef PTX_BY
}

template <int N>
__device__ __noinline__ void col(const ProbArgs& a, int j0, int pbx, int pby) {
    constexpr bool kBg = false, kCycle = true;
    const int mode_arg = COL_PROJECT;
#define PTX_BX pbx
#define PTX_BY pby
#define PTX_GX (N / RegShape<N>::C)
#include "body_col.inc"
#undef PTX_BX
#undef PTX_BY
#undef PTX_GX
}

template <int N>
__device__ __noinline__ void row_bwd(const ProbArgs& a, int j0, int nb, int pbx, int pby, int pgy) {
    constexpr int kForm = 1;
    const int mode_arg = BWD_DM, upd_obj_arg = 0, upd_probe_arg = 1;
#define PTX_BX pbx
#define PTX_BY pby
#define PTX_GY pgy
#include "body_row_bwd.inc"
#undef PTX_BX
#undef PTX_BY
#undef PTX_GY
}

// A forward-row or column item covers kPersFrames consecutive frames of one
// row band or column block (the bodies run one after the other; the block
// synchronises between them, as the next body rewrites the shared twiddles).
template <int N>
__device__ __forceinline__ void run_item(const ProbArgs& a, const PBatch& bt, int pass, int k, bool dm_fwd) {
    if (pass == 0) {
        constexpr int nbx = N / RegShape<N>::L;
        const int bx = k % nbx, f0 = (k / nbx) * kPersFrames;
        const int f1 = f0 + kPersFrames < bt.nb ? f0 + kPersFrames : bt.nb;
        for (int f = f0; f < f1; ++f) {
            if (f > f0) __syncthreads();
            if (dm_fwd)
                row_fwd<N, true>(a, bt.j0, bx, f);
            else
                row_fwd<N, false>(a, bt.j0, bx, f);
        }
    } else if (pass == 1) {
        constexpr int nbx = N / RegShape<N>::C;
        const int bx = k % nbx, f0 = (k / nbx) * kPersFrames;
        const int f1 = f0 + kPersFrames < bt.nb ? f0 + kPersFrames : bt.nb;
        for (int f = f0; f < f1; ++f) {
            if (f > f0) __syncthreads();
            col<N>(a, bt.j0, bx, f);
        }
    } else {
        constexpr int nbx = N / BwdShape<N>::L;
        row_bwd<N>(a, bt.j0, bt.nb, k % nbx, k / nbx, bt.G);
    }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

}  // namespace pers

__global__ void __launch_bounds__(kThreads, 2) k_cycle_persistent(PersArgs pa) {
    using namespace pers;
    __shared__ int s_item[3];  // segment, item within the segment, or -1
    __shared__ ProbArgs s_a;   // the item's problem, its work stack at the batch's slot
    __shared__ PBatch s_bt;
    // thread 0's view of the list: the segment of the last item (items are
    // taken in increasing order, so the search only moves forward), the batch
    // and problem whose arguments are in shared memory, and the next item index
    // (taken while the current item runs)
    int seg_at = 0, g_at = -1, prob_at = -1;
    unsigned next = 0;
    if (threadIdx.x == 0 && !*(volatile int*)&pa.ctl->abort) next = atomicAdd(&pa.ctl->head, 1u);
    for (;;) {
        if (threadIdx.x == 0) {
            int seg = -1, k = 0;
            const unsigned i = next;
            if (!*(volatile int*)&pa.ctl->abort && i < (unsigned)pa.nitems) {
                while (seg_at + 1 < pa.nseg && (unsigned)pa.seg[seg_at + 1].start <= i) ++seg_at;
                seg = seg_at;
                k = (int)(i - (unsigned)pa.seg[seg].start);
                const PSeg sg = pa.seg[seg];
                // the items this one depends on (earlier in the list)
                const unsigned* dep = nullptr;
                unsigned target = 0;
                if (sg.pass == 1) {
                    dep = &pa.done[3 * sg.g + 0];
                    target = pa.batch[sg.g].n[0];
                } else if (sg.pass == 2) {
                    dep = &pa.done[3 * sg.g + 1];
                    target = pa.batch[sg.g].n[1];
                } else if (sg.g >= kSlots) {
                    dep = &pa.done[3 * (sg.g - kSlots) + 2];
                    target = pa.batch[sg.g - kSlots].n[2];
                }
                if (dep) {
                    const long long t0 = clock64();
                    while (ld_acquire(dep) < target) {
                        if (*(volatile int*)&pa.ctl->abort || clock64() - t0 > (1ll << 31)) {
                            atomicExch(&pa.ctl->abort, 1);
                            if (pa.err_flag) {
                                *(volatile int*)pa.err_flag = 1;
                                __threadfence_system();
                            }
                            seg = -1;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                if (seg >= 0 && sg.g != g_at) {
                    s_bt = pa.batch[sg.g];
                    if (s_bt.prob != prob_at) {
                        s_a = pa.prob[s_bt.prob];
                        prob_at = s_bt.prob;
                    }
                    s_a.spec = pa.spec + (size_t)(sg.g % kSlots) * pa.slot_elems;
                    g_at = sg.g;
                }
                // the next item index, while this one runs
                if (seg >= 0) next = atomicAdd(&pa.ctl->head, 1u);
            }
            s_item[0] = seg;
            s_item[1] = k;
        }
        __syncthreads();
        const int seg = s_item[0], k = s_item[1];
        if (seg < 0) break;
        const PSeg sg = pa.seg[seg];
        const PBatch& bt = s_bt;
        const ProbArgs& a = s_a;
        const bool dm_fwd = ((pa.dm_mask >> bt.prob) & 1ull) && !pa.init;
        switch (a.N) {
            case 128: run_item<128>(a, bt, sg.pass, k, dm_fwd); break;
            case 192: run_item<192>(a, bt, sg.pass, k, dm_fwd); break;
            case 256: run_item<256>(a, bt, sg.pass, k, dm_fwd); break;
            case 384: run_item<384>(a, bt, sg.pass, k, dm_fwd); break;
            case 512: run_item<512>(a, bt, sg.pass, k, dm_fwd); break;
            default: break;
        }
        __syncthreads();  // every thread's stores of the item are issued
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&pa.done[3 * sg.g + sg.pass], 1u);
        }
    }
}

// Dynamic shared memory of the persistent kernel: the largest of its bodies.
template <int N>
constexpr size_t pers_smem_n() {
    const size_t f = sizeof(float2) * (N + (size_t)RegShape<N>::L * RegShape<N>::P);
    const size_t c = sizeof(float2) * (N + (size_t)RegShape<N>::C * RegShape<N>::P);
    using S = BwdShape<N>;
    const size_t b = sizeof(float2) * (N + (S::kRegAcc ? 2 : 1) * (size_t)S::L * N + (size_t)S::L * reg_pitch<N>()) +
                     (S::kRegAcc ? 0 : (size_t)S::L * N * (sizeof(float2) + sizeof(float)));
    return f > c ? (f > b ? f : b) : (c > b ? c : b);
}
size_t pers_smem() {
    const size_t s[] = {pers_smem_n<128>(), pers_smem_n<192>(), pers_smem_n<256>(), pers_smem_n<384>(),
                        pers_smem_n<512>()};
    size_t m = 0;
    for (size_t v : s) m = v > m ? v : m;
    return m;
}
bool pers_supported_N(int N) { return N == 128 || N == 192 || N == 256 || N == 384 || N == 512; }

cudaError_t set_attrs_persistent() {
    return cudaFuncSetAttribute(k_cycle_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pers_smem());
}
// Resident blocks of the persistent kernel on the current device (0 on error).
int pers_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cycle_persistent, kThreads, pers_smem()) != cudaSuccess)
        return 0;
    return n;
}
void launch_cycle_persistent(const PersArgs& pa, int grid, cudaStream_t s) {
    k_cycle_persistent<<<grid, kThreads, pers_smem(), s>>>(pa);
}

}  // namespace ptx
