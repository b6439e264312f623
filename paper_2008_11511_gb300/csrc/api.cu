// libptycho C ABI: argument checks, scratch layout, batch scheduling and
// CUDA-graph replay of the cycle.  The operations themselves are the kernels of
// kernels.cuh; this file only validates, lays out memory and enqueues.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/ptycho.h"
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_8();
const KernelSet* kernel_set_12();
const KernelSet* kernel_set_16();
const KernelSet* kernel_set_32();
const KernelSet* kernel_set_64();
const KernelSet* kernel_set_128();
const KernelSet* kernel_set_192();
const KernelSet* kernel_set_256();
const KernelSet* kernel_set_384();
const KernelSet* kernel_set_512();
const KernelSet* kernel_set_80();
const KernelSet* kernel_set_160();
const KernelSet* kernel_set_224();
const KernelSet* kernel_set_400();
const KernelSet* kernel_set_448();
cudaError_t set_attrs_8();
cudaError_t set_attrs_12();
cudaError_t set_attrs_16();
cudaError_t set_attrs_32();
cudaError_t set_attrs_64();
cudaError_t set_attrs_128();
cudaError_t set_attrs_192();
cudaError_t set_attrs_256();
cudaError_t set_attrs_384();
cudaError_t set_attrs_512();
cudaError_t set_attrs_80();
cudaError_t set_attrs_160();
cudaError_t set_attrs_224();
cudaError_t set_attrs_400();
cudaError_t set_attrs_448();

const KernelSet* kernel_set(int N) {
    switch (N) {
        case 8: return kernel_set_8();
        case 12: return kernel_set_12();
        case 16: return kernel_set_16();
        case 32: return kernel_set_32();
        case 64: return kernel_set_64();
        case 128: return kernel_set_128();
        case 192: return kernel_set_192();
        case 256: return kernel_set_256();
        case 384: return kernel_set_384();
        case 512: return kernel_set_512();
        case 80: return kernel_set_80();
        case 160: return kernel_set_160();
        case 224: return kernel_set_224();
        case 400: return kernel_set_400();
        case 448: return kernel_set_448();
        default: return nullptr;
    }
}

// Raise the dynamic shared-memory limit of every kernel once per device.
static cudaError_t ensure_attributes() {
    static int done_mask = 0;  // bit per device ordinal < 32
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 32 && (done_mask >> dev) & 1) return cudaSuccess;
    cudaError_t (*fns[])() = {set_attrs_8,   set_attrs_12,  set_attrs_16,  set_attrs_32,  set_attrs_64,
                              set_attrs_128, set_attrs_192, set_attrs_256, set_attrs_384, set_attrs_512,
                              set_attrs_80,  set_attrs_160, set_attrs_224, set_attrs_400, set_attrs_448,
                              set_attrs_gather_tma, set_attrs_tc, set_attrs_row_tc, set_attrs_persistent};
    for (auto f : fns)
        if ((e = f()) != cudaSuccess) return e;
    if (dev < 32) done_mask |= 1 << dev;
    return cudaSuccess;
}
}  // namespace ptx

using namespace ptx;

namespace {

thread_local std::string g_last_error;

ptx_status fail(ptx_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

}  // namespace

namespace ptx {
// Lets other translation units of the library report through ptx_last_error.
void set_last_error(const char* msg) { g_last_error = msg; }
// SMs of the current device (152 on GB300 when it cannot be asked)
int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            cudaGetLastError();
    }
    return n > 0 ? n : 152;
}
}  // namespace ptx

namespace {

ptx_status cuda_fail(cudaError_t e, const char* what) {
    return fail(PTX_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Default size of the Fourier-space batch work stack: small enough to stay
// resident in the 129 MB L2 together with the streamed exit waves.
constexpr size_t kSpecBudget = (size_t)64 << 20;
// Frames of 4 MB of spectra or more (512^2 with several modes) get a stack of
// at least kLargeFrames frames per lane instead: at 64 MB a lane would hold 5
// of them and the column pass would fill half the GPU (measured: 21.1 ->
// 20.2 ms per DM cycle of 1500 three-mode 512^2 frames).
constexpr size_t kLargeFrameBytes = (size_t)4 << 20;
constexpr size_t kLargeFrames = 21;
// Batches in flight per cycle (streams): the next batch's row passes overlap the
// current batch's column pass, and kernel tails fill in.
constexpr int kDefaultLanes = 2;
constexpr int kMaxLanes = 4;

struct Layout {
    size_t pos, mask, acc_obj, acc_probe, llk_part, maxbits, tile_ids, tile_ptr, tile_frames;
    size_t cg_obj, cg_probe, ls_part, cg;  // ML conjugate-gradient state
    size_t mbits;                          // per-thread mask bits of the register column pass
    size_t nf_t;                           // near-field transfer factors t[k] (complex64, N)
    size_t bg_acc;                         // background update sums (float, N x N)
    size_t pos_part;                       // position-shift partial sums (double, J x bands x 5)
    size_t end;
};

struct ProbHost {
    ptx_problem p;
    const KernelSet* ks = nullptr;
    int L1 = 1, C2 = 1, L3 = 1;
    int B = 1;   // frames per batch
    int G3 = 1;  // frame groups of row_bwd
    // object tiles met by at least one frame, with their frames (CSR, ascending j)
    std::vector<int> tile_ids, tile_ptr, tile_frames;
    int ntx = 0;
    int tile_h = 0;  // object tile height of the gather (0: not chosen yet)
    Layout lay{};
    ProbArgs args{};
    TileLists tiles{};
    // tensor maps of the intensities and the mask for the tensor-copy column pass (valid if tma_io)
    CUtensorMap tm_io{};
    CUtensorMap tm_mask{};
    bool tma_io = false;
    // tensor maps of Psi' and P as [J K][N][N] / [K][N][N] for the tensor-copy object gather
    CUtensorMap tm_psi3{};
    CUtensorMap tm_probe3{};
    bool tma_gather = false;
};

// Tiles of TW x TH object pixels met by at least one frame.
size_t active_tiles(const ptx_problem& p, const int32_t* positions, int TW, int TH) {
    const int ntx = (p.Wo + TW - 1) / TW, nty = (p.Ho + TH - 1) / TH;
    std::vector<char> hit((size_t)ntx * nty, 0);
    for (int j = 0; j < p.J; ++j) {
        const int r = positions[2 * j], c = positions[2 * j + 1];
        for (int ty = r / TH; ty <= (r + p.N - 1) / TH; ++ty)
            for (int tx = c / TW; tx <= (c + p.N - 1) / TW; ++tx) hit[(size_t)ty * ntx + tx] = 1;
    }
    size_t n = 0;
    for (char v : hit) n += v;
    return n;
}

// Per-tile frame lists of the object gather (host, from the positions).  The
// tile height is chosen once, at the first build: the full kObjTileH, or half
// or a quarter of it while the object has fewer tiles than two blocks per SM
// (a small object would otherwise leave most SMs idle).
void build_tiles(ProbHost& h, const int32_t* positions) {
    const ptx_problem& p = h.p;
    if (h.tile_h == 0) {
        h.tile_h = kObjTileH;
        while (h.tile_h > kObjTileH / 4 && active_tiles(p, positions, kObjTileW, h.tile_h) < 2 * 152) h.tile_h /= 2;
    }
    const int TW = kObjTileW, TH = h.tile_h;
    const int ntx = (p.Wo + TW - 1) / TW, nty = (p.Ho + TH - 1) / TH;
    std::vector<int> count((size_t)ntx * nty, 0);
    auto span = [&](int j, int& ty0, int& ty1, int& tx0, int& tx1) {
        const int r = positions[2 * j], c = positions[2 * j + 1];
        ty0 = r / TH;
        ty1 = (r + p.N - 1) / TH;
        tx0 = c / TW;
        tx1 = (c + p.N - 1) / TW;
    };
    for (int j = 0; j < p.J; ++j) {
        int ty0, ty1, tx0, tx1;
        span(j, ty0, ty1, tx0, tx1);
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) count[(size_t)ty * ntx + tx]++;
    }
    std::vector<int> slot(count.size(), -1);
    h.tile_ids.clear();
    h.tile_ptr.assign(1, 0);
    for (size_t t = 0; t < count.size(); ++t)
        if (count[t]) {
            slot[t] = (int)h.tile_ids.size();
            h.tile_ids.push_back((int)t);
            h.tile_ptr.push_back(h.tile_ptr.back() + count[t]);
        }
    h.tile_frames.assign(h.tile_ptr.back(), 0);
    std::vector<int> fill(h.tile_ids.size(), 0);
    for (int j = 0; j < p.J; ++j) {
        int ty0, ty1, tx0, tx1;
        span(j, ty0, ty1, tx0, tx1);
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) {
                const int sidx = slot[(size_t)ty * ntx + tx];
                h.tile_frames[h.tile_ptr[sidx] + fill[sidx]++] = j;
            }
    }
    h.ntx = ntx;
}

int choose_lines(int N, int K, int maxl) {
    int L = 1;
    while (K * L * 2 <= maxl && N % (L * 2) == 0) L *= 2;
    return L;
}

bool supported_N(int N) {
    static const int sizes[] = PTX_SUPPORTED_SIZES;
    for (int s : sizes)
        if (s == N) return true;
    return false;
}

ptx_status check_problem(const ptx_problem& p, int idx) {
    if (!supported_N(p.N)) return fail(PTX_ERR_UNSUPPORTED, "problem %d: frame size N=%d is not supported", idx, p.N);
    if (p.K < 1 || p.K > PTX_MAX_MODES)
        return fail(p.K < 1 ? PTX_ERR_INVALID_ARG : PTX_ERR_UNSUPPORTED, "problem %d: K=%d modes (1..%d)", idx, p.K,
                    PTX_MAX_MODES);
    if (p.J < 1) return fail(PTX_ERR_INVALID_ARG, "problem %d: J=%d must be >= 1", idx, p.J);
    if (p.Ho < p.N || p.Wo < p.N)
        return fail(PTX_ERR_INVALID_ARG, "problem %d: object %dx%d smaller than the frame %d", idx, p.Ho, p.Wo, p.N);
    if (!p.obj || !p.probe || !p.positions || !p.iobs)
        return fail(PTX_ERR_INVALID_ARG, "problem %d: obj, probe, positions and iobs must be non-null", idx);
    if ((uintptr_t)p.iobs % 16 || (uintptr_t)p.obj % 8 || (uintptr_t)p.probe % 16 || (uintptr_t)p.psi % 16)
        return fail(PTX_ERR_INVALID_ARG, "problem %d: iobs, probe and psi must be 16-byte aligned, obj 8-byte", idx);
    if (!(p.nearfield >= 0.0) || !std::isfinite(p.nearfield))
        return fail(PTX_ERR_INVALID_ARG, "problem %d: nearfield must be finite and >= 0", idx);
    if (p.nearfield > 0.0 && (p.K != 1 || p.N < 32))
        return fail(PTX_ERR_UNSUPPORTED, "problem %d: the near field needs K = 1 and N >= 32 (K=%d, N=%d)", idx, p.K,
                    p.N);
    for (int j = 0; j < p.J; ++j) {
        const int r = p.positions[2 * j], c = p.positions[2 * j + 1];
        if (r < 0 || c < 0 || r > p.Ho - p.N || c > p.Wo - p.N)
            return fail(PTX_ERR_OUT_OF_BOUNDS, "problem %d: position %d = (%d, %d) puts the %dx%d patch outside the %dx%d object",
                        idx, j, r, c, p.N, p.N, p.Ho, p.Wo);
    }
    return PTX_OK;
}

// Batches of frames: `lanes` batches are in flight at once (one per stream),
// each with its own slice of the work-stack region of `spec_bytes`.

void set_batch(ProbHost& h, size_t spec_bytes, int lanes, int cap = 0, int slots = 0) {
    const ptx_problem& p = h.p;
    const size_t frame_bytes = (size_t)p.K * p.N * p.N * sizeof(float2);
    size_t B = (spec_bytes / lanes) / 256 * 256 / frame_bytes;
    if (cap > 0 && B > (size_t)cap) B = cap;
    if (B < 1) B = 1;
    if (B > (size_t)p.J) B = p.J;
    if (B > 32768) B = 32768;  // grid.y limit of the batch kernels
    h.B = (int)B;
    // frame slots G of the row-backward pass: (N / L3) row blocks x K modes x G
    // blocks, as many as are resident at once (each block loops over its
    // frames and flushes its probe sums once)
    int per_sm = h.ks->row_bwd_per_sm();
    if (per_sm <= 0) per_sm = 2;
    const int resident = per_sm * sm_count();
    const int rowblk = p.N / h.L3 * p.K;
    int G = slots > 0 ? slots : resident / rowblk;
    if (G > h.B) G = h.B;
    if (G < 1) G = 1;
    h.G3 = G;
}

void plan_problem(ProbHost& h) {
    const ptx_problem& p = h.p;
    h.ks = kernel_set(p.N);
    const int maxl = h.ks->max_lines;
    if (use_reg_kernels(h.ks, p.K)) {
        h.L1 = h.L3 = h.ks->reg_lines;
        // LLK partials per frame: one per column block (near field: per row
        // block of its projection pass)
        h.C2 = p.nearfield > 0.0 ? h.ks->reg_lines : h.ks->reg_cols;
    } else {
        h.L1 = choose_lines(p.N, p.K, maxl);
        h.C2 = choose_lines(p.N, p.K, maxl);
        h.L3 = choose_lines(p.N, p.K, maxl);
    }
    const size_t frame_bytes = (size_t)p.K * p.N * p.N * sizeof(float2);
    size_t budget = kSpecBudget;
    if (frame_bytes >= kLargeFrameBytes) budget = std::max(budget, kDefaultLanes * kLargeFrames * frame_bytes);
    set_batch(h, budget, kDefaultLanes);
}

// Per-problem regions (offsets relative to the problem's base).
size_t layout_problem(ProbHost& h) {
    const ptx_problem& p = h.p;
    size_t o = 0;
    h.lay.pos = o;
    o = align_up(o + sizeof(int2) * (size_t)p.J);
    h.lay.mask = o;
    o = align_up(o + (size_t)p.N * p.N);
    h.lay.acc_obj = o;
    o = align_up(o + sizeof(float4) * (size_t)p.Ho * p.Wo);
    h.lay.acc_probe = o;
    o = align_up(o + sizeof(float4) * (size_t)p.K * p.N * p.N);
    h.lay.llk_part = o;
    o = align_up(o + sizeof(double) * (size_t)p.J * (p.N / h.C2));
    h.lay.maxbits = o;
    o = align_up(o + 2 * sizeof(unsigned));
    // tile lists sized for any positions (ptx_set_positions rewrites them in place):
    // every object tile, and per frame the tiles an N x N patch can meet
    const int th = h.tile_h > 0 ? h.tile_h : kObjTileH / 4;
    const size_t ntiles_max = (size_t)((p.Wo + kObjTileW - 1) / kObjTileW) * ((p.Ho + th - 1) / th);
    const size_t per_frame = (size_t)((p.N + th - 1) / th + 1) * ((p.N + kObjTileW - 1) / kObjTileW + 1);
    h.lay.tile_ids = o;
    o = align_up(o + sizeof(int) * std::max(h.tile_ids.size(), ntiles_max));
    h.lay.tile_ptr = o;
    o = align_up(o + sizeof(int) * std::max(h.tile_ptr.size(), ntiles_max + 1));
    h.lay.tile_frames = o;
    o = align_up(o + sizeof(int) * std::max(h.tile_frames.size(), (size_t)p.J * per_frame));
    h.lay.pos_part = o;
    o = align_up(o + 5 * sizeof(double) * (size_t)p.J * ((p.N + 7) / 8));
    // CG: gradient, previous gradient and direction of object and probe
    h.lay.cg_obj = o;
    o = align_up(o + 3 * sizeof(float2) * (size_t)p.Ho * p.Wo);
    h.lay.cg_probe = o;
    o = align_up(o + 3 * sizeof(float2) * (size_t)p.K * p.N * p.N);
    h.lay.ls_part = o;
    o = align_up(o + 2 * sizeof(double) * (size_t)p.J * (p.N / ls_cols(h.ks, p.K)));
    h.lay.cg = o;
    o = align_up(o + (8 + 3 * (size_t)kCgBlocks) * sizeof(double));  // scalars, then the dot-product partials
    h.lay.mbits = o;
    if (use_reg_kernels(h.ks, p.K)) o = align_up(o + sizeof(uint32_t) * (size_t)(p.N / h.ks->reg_cols) * kThreads);
    h.lay.nf_t = o;
    if (p.nearfield > 0.0) o = align_up(o + sizeof(float2) * (size_t)p.N);
    h.lay.bg_acc = o;
    if (p.background) o = align_up(o + sizeof(float) * (size_t)p.N * p.N);
    h.lay.end = o;
    return o;
}

struct GraphKey {
    std::vector<int> algos;
    uint32_t flags;
    int lanes;
    int tma;
    bool operator<(const GraphKey& o) const {
        if (flags != o.flags) return flags < o.flags;
        if (lanes != o.lanes) return lanes < o.lanes;
        if (tma != o.tma) return tma < o.tma;
        return algos < o.algos;
    }
};

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// Row-major [h][w] array of `es`-byte elements (8: complex64 moved as 64-bit
// words, 4: float32, 1: bytes), copied in boxes of bh rows x bw elements.
bool encode_2d(CUtensorMap* m, int es, const void* base, uint64_t w, uint64_t h, uint32_t bw, uint32_t bh) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const CUtensorMapDataType dt = es == 8   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                             : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    cuuint64_t dims[2] = {w, h};
    cuuint64_t strides[1] = {w * es};
    cuuint32_t box[2] = {bw, bh};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, dt, 2, (void*)base, dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Complex64 array [d][h][w] (moved as 64-bit words) in boxes of bh x bw x 1;
// reads outside the array fill with zeros.
bool encode_3d(CUtensorMap* m, const void* base, uint64_t w, uint64_t h, uint64_t d, uint32_t bw, uint32_t bh) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {w, h, d};
    cuuint64_t strides[2] = {w * 8, w * h * 8};
    cuuint32_t box[3] = {bw, bh, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, (void*)base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

struct ptx_handle {
    std::vector<ProbHost> probs;
    char* scratch = nullptr;
    size_t scratch_bytes = 0;
    size_t spec_off = 0, ctl_off = 0;
    Ctl* ctl = nullptr;
    double alpha_obj = 1e-2, alpha_probe = 1e-2;
    int device = 0;
    cudaStream_t cap_stream = nullptr;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::map<GraphKey, int64_t> graph_kernels;  // kernel nodes of each captured cycle
    // batch lanes: extra streams and fork / join events (lane 0 is the call's stream)
    int lanes = kDefaultLanes;
    int batch_cap = 0;  // ptx_set_param "batch_frames"
    int bwd_slots = 0;  // ptx_set_param "bwd_slots": frame slots of the row-backward pass (0: by occupancy)
    // ptx_set_param "persistent": the batch passes of all problems as one persistent launch
    int persistent = 0;
    size_t pers_off = 0;
    bool pers_dirty = true;  // tables to rebuild and upload before the next cycle
    int pers_selftest = 0;   // ptx_set_param "persistent_selftest": a dependency that is never met
    int tc_selftest = 0;     // ptx_set_param "tc_selftest": a tensor-core stage whose commit never comes
    int tc_rows = 0;         // ptx_set_param "tc_rows": the row passes' DFT stages on the tensor cores too
    int pdl = 1;             // ptx_set_param "pdl": batch passes launched as programmatic dependents
    int pers_nitems = 0, pers_nseg = 0, pers_nbatch = 0;
    std::vector<ProbArgs> pers_prob;
    std::vector<PSeg> pers_seg;
    std::vector<PBatch> pers_batch;
    int tma = 0;        // ptx_set_param "tma": column pass fed by tensor copies where available
    int tma_gather = 1; // ptx_set_param "tma_gather": object gather fed by tensor copies where available
    int tc = 0;         // ptx_set_param "tc": TcForm of the column pass's DFT stages on the tensor cores (N = 256, K = 1)
    // flag in mapped pinned host memory that a device wait sets when it gives up
    int* err_host = nullptr;
    int* err_dev = nullptr;
    size_t spec_bytes = 0;
    cudaStream_t lane_stream[kMaxLanes] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kMaxLanes] = {};
    std::vector<cudaEvent_t> prob_ev;  // [problem][lane]: a problem's batches done on a lane
    // per-kernel timing (ptx_profile_enable)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_used;  // (kind, index of the start event in ev_pool)
};

namespace {

// Mask bits of the register column pass: entry [xb][t] holds, for thread t of
// column block xb, bit (i M + k1) = mask at row k2 + R k1, column xb C + c of its
// pass-2 item i (w = t + 256 i, k2 = w / C, c = w % C), C = columns per block.
std::vector<uint32_t> mask_bits(const KernelSet* ks, int N, const uint8_t* mask) {
    const int C = ks->reg_cols, R = ks->R, M = ks->M, XB = N / C;
    const int I2 = (C * R + kThreads - 1) / kThreads;
    std::vector<uint32_t> t((size_t)XB * kThreads, 0u);
    for (int xb = 0; xb < XB; ++xb)
        for (int th = 0; th < kThreads; ++th) {
            uint32_t bits = 0u;
            for (int i = 0; i < I2; ++i) {
                const int w = th + i * kThreads;
                if (w >= C * R) continue;
                const int k2 = w / C, c = w % C;
                for (int k1 = 0; k1 < M; ++k1)
                    if (mask[(size_t)(k2 + R * k1) * N + xb * C + c]) bits |= 1u << (i * M + k1);
            }
            t[(size_t)xb * kThreads + th] = bits;
        }
    return t;
}

// Region of the persistent schedule's tables (after the control block): the
// problems' arguments, the segments and batches of the work list, the item
// counter and the per-(batch, pass) done counters, sized for batches of one
// frame (the most batches any schedule can have).
struct PersLayout {
    size_t prob = 0, seg = 0, batch = 0, ctl = 0, done = 0, end = 0;
    size_t max_batches = 0;
};
PersLayout pers_layout(size_t base, size_t nprob, size_t frames) {
    PersLayout L;
    L.max_batches = frames;
    size_t o = base;
    L.prob = o;
    o = align_up(o + sizeof(ProbArgs) * nprob);
    L.seg = o;
    o = align_up(o + sizeof(PSeg) * 3 * frames);
    L.batch = o;
    o = align_up(o + sizeof(PBatch) * frames);
    L.ctl = o;
    o = align_up(o + sizeof(PCtl));
    L.done = o;
    o = align_up(o + sizeof(unsigned) * 3 * frames);
    L.end = o;
    return L;
}

ptx_status compute_layout(std::vector<ProbHost>& probs, size_t* spec_off, size_t* ctl_off, size_t* total,
                          size_t* pers_off = nullptr) {
    size_t o = 0;
    size_t spec = 0;
    size_t frames = 0;
    for (auto& h : probs) {
        plan_problem(h);
        size_t sz = layout_problem(h);
        // shift this problem's regions to its base
        h.lay.pos += o;
        h.lay.mask += o;
        h.lay.acc_obj += o;
        h.lay.acc_probe += o;
        h.lay.llk_part += o;
        h.lay.maxbits += o;
        h.lay.tile_ids += o;
        h.lay.tile_ptr += o;
        h.lay.tile_frames += o;
        h.lay.cg_obj += o;
        h.lay.cg_probe += o;
        h.lay.ls_part += o;
        h.lay.cg += o;
        h.lay.mbits += o;
        h.lay.nf_t += o;
        h.lay.bg_acc += o;
        h.lay.pos_part += o;
        h.lay.end += o;
        o += sz;
        size_t s = (size_t)h.B * kDefaultLanes * h.p.K * h.p.N * h.p.N * sizeof(float2);
        if (s > spec) spec = s;
        frames += (size_t)h.p.J;
    }
    *ctl_off = o;
    o = align_up(o + sizeof(Ctl));
    if (pers_off) *pers_off = o;
    o = pers_layout(o, probs.size(), frames).end;
    *spec_off = o;
    o = align_up(o + spec);
    *total = o;
    return PTX_OK;
}

void fill_args(ptx_handle* h, ProbHost& ph) {
    ProbArgs& a = ph.args;
    const ptx_problem& p = ph.p;
    a.N = p.N;
    a.K = p.K;
    a.J = p.J;
    a.Ho = p.Ho;
    a.Wo = p.Wo;
    a.obj = (float2*)p.obj;
    a.probe = (float2*)p.probe;
    a.iobs = p.iobs;
    a.psi = (float2*)p.psi;
    a.pos = (const int2*)(h->scratch + ph.lay.pos);
    a.mask = (const uint8_t*)(h->scratch + ph.lay.mask);
    a.acc_obj = (float4*)(h->scratch + ph.lay.acc_obj);
    a.acc_probe = (float4*)(h->scratch + ph.lay.acc_probe);
    a.spec = (float2*)(h->scratch + h->spec_off);
    a.llk_part = (double*)(h->scratch + ph.lay.llk_part);
    a.maxbits = (unsigned*)(h->scratch + ph.lay.maxbits);
    a.grad_obj = nullptr;
    a.grad_probe = nullptr;
    a.L1 = ph.L1;
    a.C2 = ph.C2;
    a.L3 = ph.L3;
    a.dir_obj = nullptr;
    a.dir_probe = nullptr;
    a.ls_part = (double*)(h->scratch + ph.lay.ls_part);
    a.err_flag = h->err_dev;
    a.mbits = (const uint32_t*)(h->scratch + ph.lay.mbits);
    a.nf_t = ph.p.nearfield > 0.0 ? (const float2*)(h->scratch + ph.lay.nf_t) : nullptr;
    a.bg = ph.p.background;
    a.bg_acc = nullptr;  // set only for the column passes of AP cycles that update the background
    ph.tiles.tile_ids = (const int*)(h->scratch + ph.lay.tile_ids);
    ph.tiles.tile_ptr = (const int*)(h->scratch + ph.lay.tile_ptr);
    ph.tiles.tile_frames = (const int*)(h->scratch + ph.lay.tile_frames);
    ph.tiles.ntx = ph.ntx;
    ph.tiles.th = ph.tile_h;
}

// Second half of Psi2ObjProbe, in stages: probe normalisation from its
// accumulators; object numerator / denominator gathered from Psi' with the
// current (new) probe; object normalisation.
enum Stage { STAGE_PROBE = 0x100, STAGE_OBJ_GATHER = 0x200, STAGE_OBJ_NORMALISE = 0x400 };

enum Algo { ALGO_AP = 0, ALGO_DM = 1 };

// Whether the register batch passes of a problem go out as programmatic
// dependents of the pass before them on the same stream: far field, no
// background, not while profiling (whose events sit between the launches).
// The caller launches the first forward pass of a stream plainly.
bool pass_pdl(const ptx_handle* h, const ProbHost& ph) {
    return h->pdl && !h->profiling && ph.p.nearfield <= 0.0 && !ph.p.background && use_reg_kernels(ph.ks, ph.p.K);
}

// Bracket one launch with profiling events when profiling is on.
struct ProfScope {
    ptx_handle* h;
    int kind;
    cudaStream_t s;
    int idx = -1;
    ProfScope(ptx_handle* h_, int kind_, cudaStream_t s_) : h(h_), kind(kind_), s(s_) {
        if (!h->profiling) return;
        idx = (int)h->ev_used.size() * 2;
        while ((int)h->ev_pool.size() < idx + 2) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) {
                idx = -1;
                return;
            }
            h->ev_pool.push_back(e);
        }
        cudaEventRecord(h->ev_pool[idx], s);
    }
    ~ProfScope() {
        if (idx < 0) return;
        cudaEventRecord(h->ev_pool[idx + 1], s);
        h->ev_used.push_back({kind, idx});
    }
};

void enqueue_stages(ptx_handle* h, ProbHost& ph, int stages, cudaStream_t s) {
    const ProbArgs& a = ph.args;
    if (stages & STAGE_PROBE) {
        {
            ProfScope ps(h, PTX_KERNEL_DEN_MAX, s);
            k_den_max<<<2 * 152, 256, 0, s>>>(a, 0, 1);
        }
        ProfScope ps(h, PTX_KERNEL_NORMALISE, s);
        k_normalise<<<4 * 152, 256, 0, s>>>(a, (float)h->alpha_obj, (float)h->alpha_probe, 0, 1);
    }
    // gather and normalisation in one call: the gather also takes max D_O;
    // otherwise (accumulators summed across ranks in between) a separate pass does
    const bool fused_max = (stages & STAGE_OBJ_GATHER) && (stages & STAGE_OBJ_NORMALISE);
    if ((stages & STAGE_OBJ_GATHER) && !ph.tile_ids.empty()) {
        ProfScope ps(h, PTX_KERNEL_OBJ_GATHER, s);
        if (h->tma_gather && ph.tma_gather)
            launch_obj_gather_tma(&ph.tm_psi3, &ph.tm_probe3, a, ph.tiles, (int)ph.tile_ids.size(), fused_max ? 1 : 0, s);
        else
            k_obj_gather<<<(unsigned)ph.tile_ids.size(), 256, 0, s>>>(a, ph.tiles, fused_max ? 1 : 0);
    }
    if (stages & STAGE_OBJ_NORMALISE) {
        if (!fused_max) {
            ProfScope ps(h, PTX_KERNEL_DEN_MAX, s);
            k_den_max<<<2 * 152, 256, 0, s>>>(a, 1, 0);
        }
        ProfScope ps(h, PTX_KERNEL_NORMALISE, s);
        k_normalise<<<4 * 152, 256, 0, s>>>(a, (float)h->alpha_obj, (float)h->alpha_probe, 1, 0);
    }
}

ptx_status ensure_lanes(ptx_handle* h) {
    cudaError_t e;
    if (!h->fork_ev && (e = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "cudaEventCreate");
    while (h->prob_ev.size() < h->probs.size() * kMaxLanes) {
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate");
        h->prob_ev.push_back(ev);
    }
    for (int l = 0; l < kMaxLanes; ++l) {
        if (!h->lane_stream[l] &&
            (e = cudaStreamCreateWithFlags(&h->lane_stream[l], cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreateWithFlags");
        if (!h->join_ev[l] && (e = cudaEventCreateWithFlags(&h->join_ev[l], cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate");
    }
    return PTX_OK;
}

// The persistent schedule serves handles whose problems all run the
// register-resident one-mode far-field passes of its sizes, without a
// background; other handles keep the per-batch launches.
bool pers_eligible(const ptx_handle* h) {
    if (h->probs.empty() || h->probs.size() > 64) return false;
    const size_t slot_bytes = (h->spec_bytes / kPersSlots) / 256 * 256;
    for (const ProbHost& ph : h->probs) {
        if (!pers_supported_N(ph.p.N) || ph.p.K != 1 || ph.p.nearfield > 0.0 || ph.p.background) return false;
        if (slot_bytes < (size_t)ph.p.N * ph.p.N * sizeof(float2)) return false;  // a slot holds a frame
    }
    return true;
}

// Work list of the persistent schedule (host): the batches of every problem
// (work-stack slots of a third of the stack each), and the segments of their
// items in pipeline order — step s: forward items of batch s, column items of
// s - 1, backward items of s - 2.
void pers_build(ptx_handle* h) {
    const size_t slot_bytes = (h->spec_bytes / kPersSlots) / 256 * 256;
    h->pers_prob.clear();
    h->pers_seg.clear();
    h->pers_batch.clear();
    for (size_t pi = 0; pi < h->probs.size(); ++pi) {
        const ProbHost& ph = h->probs[pi];
        const ptx_problem& p = ph.p;
        h->pers_prob.push_back(ph.args);
        size_t B = slot_bytes / ((size_t)p.N * p.N * sizeof(float2));
        if (h->batch_cap > 0 && B > (size_t)h->batch_cap) B = h->batch_cap;
        B = std::max<size_t>(1, std::min<size_t>(B, (size_t)p.J));
        const int L = ph.ks->reg_lines, C = ph.ks->reg_cols;
        int per_sm = ph.ks->row_bwd_per_sm();
        if (per_sm <= 0) per_sm = 2;
        const int G0 = h->bwd_slots > 0 ? h->bwd_slots : std::max(1, per_sm * sm_count() / (p.N / L));
        for (int j0 = 0; j0 < p.J; j0 += (int)B) {
            const int nb = (int)std::min<size_t>(B, (size_t)(p.J - j0));
            const int G = std::min(G0, nb);
            PBatch bt{};
            bt.prob = (int)pi;
            bt.j0 = j0;
            bt.nb = nb;
            bt.G = G;
            const int fgroups = (nb + kPersFrames - 1) / kPersFrames;  // frames per row / column item
            bt.n[0] = (unsigned)((p.N / L) * fgroups);
            bt.n[1] = (unsigned)((p.N / C) * fgroups);
            bt.n[2] = (unsigned)((p.N / L) * G);
            h->pers_batch.push_back(bt);
        }
    }
    const int nbatch = (int)h->pers_batch.size();
    // self-test of the bounded waits: batch 0's column items wait for one
    // forward item more than there are, so their wait runs out
    if (h->pers_selftest && nbatch > 0) h->pers_batch[0].n[0] += 1;
    long long start = 0;
    for (int st = 0; st < nbatch + 2; ++st)
        for (int pass = 0; pass < 3; ++pass) {
            const int g = st - pass;
            if (g < 0 || g >= nbatch) continue;
            h->pers_seg.push_back(PSeg{g, pass, (int)start, 0});
            start += h->pers_batch[g].n[pass] - (h->pers_selftest && g == 0 && pass == 0 ? 1 : 0);
        }
    h->pers_nbatch = nbatch;
    h->pers_nseg = (int)h->pers_seg.size();
    h->pers_nitems = (int)start;
}

// Upload the tables (before the cycle's graph is launched; outside any capture).
ptx_status pers_upload(ptx_handle* h, cudaStream_t s) {
    size_t frames = 0;
    for (const ProbHost& ph : h->probs) frames += (size_t)ph.p.J;
    const PersLayout L = pers_layout(h->pers_off, h->probs.size(), frames);
    pers_build(h);
    if ((size_t)h->pers_nbatch > L.max_batches) return fail(PTX_ERR_NOT_READY, "persistent work list too long");
    cudaError_t e = cudaMemcpyAsync(h->scratch + L.prob, h->pers_prob.data(), sizeof(ProbArgs) * h->pers_prob.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->scratch + L.seg, h->pers_seg.data(), sizeof(PSeg) * h->pers_seg.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->scratch + L.batch, h->pers_batch.data(), sizeof(PBatch) * h->pers_batch.size(),
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "uploading the persistent work list");
    h->pers_dirty = false;
    return PTX_OK;
}

// The batch passes of every problem as one persistent launch, after zeroing its counters.
void enqueue_persistent(ptx_handle* h, const std::vector<int>& algos, bool init, cudaStream_t s) {
    size_t frames = 0;
    for (const ProbHost& ph : h->probs) frames += (size_t)ph.p.J;
    const PersLayout L = pers_layout(h->pers_off, h->probs.size(), frames);
    cudaMemsetAsync(h->scratch + L.ctl, 0, L.end - L.ctl, s);
    PersArgs pa{};
    pa.seg = (const PSeg*)(h->scratch + L.seg);
    pa.nseg = h->pers_nseg;
    pa.nitems = h->pers_nitems;
    pa.batch = (const PBatch*)(h->scratch + L.batch);
    pa.nbatch = h->pers_nbatch;
    pa.prob = (const ProbArgs*)(h->scratch + L.prob);
    pa.spec = (float2*)(h->scratch + h->spec_off);
    pa.slot_elems = (h->spec_bytes / kPersSlots) / 256 * 256 / sizeof(float2);
    pa.ctl = (PCtl*)(h->scratch + L.ctl);
    pa.done = (unsigned*)(h->scratch + L.done);
    pa.err_flag = h->err_dev;
    pa.dm_mask = 0;
    for (size_t i = 0; i < algos.size(); ++i)
        if (algos[i] == ALGO_DM) pa.dm_mask |= 1ull << i;
    pa.init = init ? 1 : 0;
    const int per_sm = std::max(1, pers_blocks_per_sm());
    ProfScope ps(h, PTX_KERNEL_ROW_FWD, s);
    launch_cycle_persistent(pa, per_sm * sm_count(), s);
}

// Number format of the column pass's DFT stages for a call: a PTX_FORM_* flag,
// else the handle's "tc" parameter.
int tc_form(const ptx_handle* h, uint32_t flags) {
    if (flags & PTX_FORM_TF32X2) return TC_TF32X2;
    if (flags & PTX_FORM_BF16X3) return TC_BF16X3;
    if (flags & PTX_FORM_BF16X2) return TC_BF16X2;
    return h->tc;
}

// One cycle of every problem, enqueued on `s`.  With one lane everything runs
// on s.  With several, the batches of all problems go round-robin to the lane
// streams, each lane with its own slice of the work-stack region; s forks the
// lanes, waits for a problem's batches before running that problem's overlap
// update and LLK reduction (while the lanes go on with the next problem), and
// joins the lanes at the end.
ptx_status enqueue_cycle(ptx_handle* h, const std::vector<int>& algos, uint32_t flags, cudaStream_t s) {
    const int form = tc_form(h, flags);
    const bool upd_o = flags & PTX_UPDATE_OBJ;
    const bool upd_p = flags & PTX_UPDATE_PROBE;
    const bool init = flags & PTX_DM_INIT_PSI;
    const int np = (int)h->probs.size();
    const int lanes = h->profiling ? 1 : h->lanes;  // per-kernel timing wants kernels alone
    const bool pers = h->persistent && !h->profiling && pers_eligible(h) && !(flags & PTX_UPDATE_BACKGROUND) &&
                      form == TC_NONE;
    if (pers) {
        enqueue_persistent(h, algos, init, s);
        for (int pi = 0; pi < np; ++pi) {
            ProbHost& ph = h->probs[pi];
            const ProbArgs& a = ph.args;
            if (!(flags & PTX_NO_NORMALISE))
                enqueue_stages(h, ph, (upd_p ? STAGE_PROBE : 0) | (upd_o ? STAGE_OBJ_GATHER | STAGE_OBJ_NORMALISE : 0),
                               s);
            ProfScope ps(h, PTX_KERNEL_CYCLE_END, s);
            k_cycle_end<<<kCycleEndBlocks, 256, 0, s>>>(h->ctl, a, pi, a.N / a.C2, pi == np - 1);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        return PTX_OK;
    }
    if (lanes > 1) {
        ptx_status st = ensure_lanes(h);
        if (st != PTX_OK) return st;
        cudaEventRecord(h->fork_ev, s);
        for (int l = 0; l < lanes; ++l) cudaStreamWaitEvent(h->lane_stream[l], h->fork_ev, 0);
    }
    // lane slices of the work stack, in elements, 256-byte aligned
    const size_t slice = (h->spec_bytes / lanes) / 256 * 256 / sizeof(float2);
    int next_lane = 0;
    for (int pi = 0; pi < np; ++pi) {
        ProbHost& ph = h->probs[pi];
        set_batch(ph, h->spec_bytes, lanes, h->batch_cap, h->bwd_slots);
        const ProbArgs& a = ph.args;
        const KernelSet* ks = ph.ks;
        const int algo = algos[pi];
        const bool upd_bg = (flags & PTX_UPDATE_BACKGROUND) && algo == ALGO_AP && ph.p.background;
        const int fwd_mode = (algo == ALGO_DM && !init) ? X_DM : X_PHI;
        const int bwd_mode = (algo == ALGO_DM) ? BWD_DM : BWD_AP;
        // the row passes' DFT stages on the tensor cores (with a tensor-core form,
        // "tc_rows": 256^2 frames of one mode and 512^2 frames of any number of
        // modes, far field, without a background)
        const bool tc_rows = form != TC_NONE && h->tc_rows && ((ph.p.N == 256 && ph.p.K == 1) || ph.p.N == 512) &&
                             ph.p.nearfield <= 0.0 && !ph.p.background;
        bool used[kMaxLanes] = {};
        // programmatic dependent launches of the FP32 register passes, each after
        // another of them on the same lane (the first forward pass of a lane
        // follows event waits or the previous problem's kernels)
        const bool tc_col = form != TC_NONE && ((ph.p.N == 256 && ph.p.K == 1) || ph.p.N == 512) &&
                            !ph.p.background;
        // (one mode: with several modes the dependents waiting beside the other
        // lane's blocks cost more than they save, 20.15 -> 20.21 ms at 512^2, K = 3)
        const bool pdl = pass_pdl(h, ph) && !tc_col && ph.p.K == 1;
        for (int j0 = 0; j0 < ph.p.J; j0 += ph.B) {
            const int nb = std::min(ph.B, ph.p.J - j0);
            const int G = std::min(ph.G3, nb);
            const int lane = next_lane;
            next_lane = (next_lane + 1) % lanes;
            const bool pdl_fwd = pdl && used[lane];
            used[lane] = true;
            cudaStream_t ls = lanes == 1 ? s : h->lane_stream[lane];
            ProbArgs al = a;
            al.spec = a.spec + lane * slice;
            if (upd_bg) al.bg_acc = (float*)(h->scratch + ph.lay.bg_acc);
            {
                ProfScope ps(h, PTX_KERNEL_ROW_FWD, ls);
                if (tc_rows)
                    launch_row_fwd_tc(al, j0, nb, fwd_mode == X_DM, form, ls);
                else
                    ks->row_fwd(al, j0, nb, fwd_mode, ls, pdl_fwd);
            }
            bool col_plain = true;  // the column pass is the register kernel (not the tensor-copy one)
            if (ph.p.nearfield > 0.0) {
                // propagate, project at the detector, propagate back
                {
                    ProfScope ps(h, PTX_KERNEL_COL, ls);
                    ks->col_nf(al, nb, +1, ls);
                }
                {
                    ProfScope ps(h, PTX_KERNEL_COL, ls);
                    ks->row_proj(al, j0, nb, 0, ls);
                }
                {
                    ProfScope ps(h, PTX_KERNEL_COL, ls);
                    ks->col_nf(al, nb, -1, ls);
                }
            } else if (tc_col) {
                ProfScope ps(h, PTX_KERNEL_COL, ls);
                launch_col_tc(al, j0, nb, form, h->tc_selftest, ls);
            } else {
                ProfScope ps(h, PTX_KERNEL_COL, ls);
                CUtensorMap tm_spec;
                const int grid = (h->tma && ph.tma_io && ks->col_tma && !ph.p.background) ? ks->col_tma_grid() : 0;
                if (grid > 0 && encode_2d(&tm_spec, 8, al.spec, ph.p.N, (uint64_t)ph.B * ph.p.N,
                                          (uint32_t)ks->reg_lines, (uint32_t)ph.p.N)) {
                    ks->col_tma(&tm_spec, &ph.tm_io, &ph.tm_mask, al, j0, nb, grid, ls);
                    col_plain = false;
                } else {
                    ks->col(al, j0, nb, COL_PROJECT, ls, pdl);
                }
            }
            {
                ProfScope ps(h, PTX_KERNEL_ROW_BWD, ls);
                if (tc_rows)
                    launch_row_bwd_tc(al, j0, nb, G, upd_p ? 1 : 0, form, ls);
                else
                    ks->row_bwd(al, j0, nb, G, bwd_mode, 0, upd_p, ls, pdl && col_plain);
            }
        }
        if (lanes > 1)
            for (int l = 0; l < lanes; ++l)
                if (used[l]) {
                    cudaEvent_t ev = h->prob_ev[(size_t)pi * kMaxLanes + l];
                    cudaEventRecord(ev, h->lane_stream[l]);
                    cudaStreamWaitEvent(s, ev, 0);
                }
        if (upd_bg) k_bg_update<<<2 * 152, 256, 0, s>>>(ph.p.background, (float*)(h->scratch + ph.lay.bg_acc),
                                                        (const uint8_t*)(h->scratch + ph.lay.mask), ph.p.N * ph.p.N,
                                                        1.0f / (float)ph.p.J);
        if (!(flags & PTX_NO_NORMALISE))
            enqueue_stages(h, ph, (upd_p ? STAGE_PROBE : 0) | (upd_o ? STAGE_OBJ_GATHER | STAGE_OBJ_NORMALISE : 0), s);
        ProfScope ps(h, PTX_KERNEL_CYCLE_END, s);
        k_cycle_end<<<kCycleEndBlocks, 256, 0, s>>>(h->ctl, a, pi, a.N / a.C2, pi == np - 1);
    }
    if (lanes > 1)
        for (int l = 0; l < lanes; ++l) {
            cudaEventRecord(h->join_ev[l], h->lane_stream[l]);
            cudaStreamWaitEvent(s, h->join_ev[l], 0);
        }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return PTX_OK;
}

ptx_status get_graph(ptx_handle* h, const std::vector<int>& algos, uint32_t flags, cudaGraphExec_t* out) {
    GraphKey key{algos, flags, h->lanes, h->tma | (h->tma_gather << 1) | (h->tc << 2)};
    auto it = h->graphs.find(key);
    if (it != h->graphs.end()) {
        *out = it->second;
        return PTX_OK;
    }
    cudaError_t e;
    if (!h->cap_stream) {
        if ((e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    if (h->lanes > 1) {
        ptx_status st0 = ensure_lanes(h);
        if (st0 != PTX_OK) return st0;
    }
    if ((e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamBeginCapture");
    ptx_status st = enqueue_cycle(h, algos, flags, h->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->cap_stream, &g);
    if (st != PTX_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    {
        size_t n = 0;
        int64_t nk = 0;
        if (cudaGraphGetNodes(g, nullptr, &n) == cudaSuccess && n > 0) {
            std::vector<cudaGraphNode_t> nodes(n);
            if (cudaGraphGetNodes(g, nodes.data(), &n) == cudaSuccess)
                for (size_t i = 0; i < n; ++i) {
                    cudaGraphNodeType t;
                    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
                }
        }
        h->graph_kernels[key] = nk;
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    h->graphs[key] = ex;
    *out = ex;
    return PTX_OK;
}

void drop_graphs(ptx_handle* h) {
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    h->graph_kernels.clear();
}

ptx_status check_device(ptx_handle* h) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != h->device)
        return fail(PTX_ERR_INVALID_ARG, "handle was created on device %d but device %d is current", h->device, dev);
    return PTX_OK;
}

ptx_status run_cycles(ptx_handle* h, const std::vector<int>& algos, int ncycles, uint32_t flags, double* llk_dev,
                      void* stream) {
    if (!h) return fail(PTX_ERR_INVALID_ARG, "null handle");
    if (ncycles < 0) return fail(PTX_ERR_INVALID_ARG, "ncycles=%d must be >= 0", ncycles);
    const uint32_t forms = PTX_FORM_TF32X2 | PTX_FORM_BF16X3 | PTX_FORM_BF16X2;
    const uint32_t known = PTX_UPDATE_OBJ | PTX_UPDATE_PROBE | PTX_DM_INIT_PSI | PTX_NO_NORMALISE | PTX_NO_GRAPH |
                           PTX_UPDATE_BACKGROUND | forms;
    if (flags & ~known) return fail(PTX_ERR_INVALID_ARG, "unknown flag bits 0x%x", flags & ~known);
    if (__builtin_popcount(flags & forms) > 1) return fail(PTX_ERR_INVALID_ARG, "more than one PTX_FORM_* flag");
    if ((int)algos.size() != (int)h->probs.size()) return fail(PTX_ERR_INVALID_ARG, "one algorithm per problem");
    for (int a : algos)
        if (a != ALGO_AP && a != ALGO_DM) return fail(PTX_ERR_INVALID_ARG, "algorithm %d is neither AP nor DM", a);
    if (flags & PTX_UPDATE_BACKGROUND)
        for (size_t i = 0; i < algos.size(); ++i)
            if (algos[i] != ALGO_AP && h->probs[i].p.background)
                return fail(PTX_ERR_INVALID_ARG, "problem %zu: the background is updated in AP cycles only", i);
    for (size_t i = 0; i < h->probs.size(); ++i)
        if (!h->probs[i].p.psi)
            return fail(PTX_ERR_INVALID_ARG, "problem %zu: AP and DM cycles need the psi array", i);
    ptx_status st = check_device(h);
    if (st != PTX_OK) return st;
    if (h->err_host && *(volatile int*)h->err_host) {
        *(volatile int*)h->err_host = 0;
        return fail(PTX_ERR_TIMEOUT, "a bounded device wait of an earlier call gave up (its results are invalid)");
    }
    if (ncycles == 0) return PTX_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->persistent && h->pers_dirty && pers_eligible(h)) {
        drop_graphs(h);  // they hold the old work list's sizes
        if ((st = pers_upload(h, s)) != PTX_OK) return st;
    }
    k_set_ctl<<<1, 1, 0, s>>>(h->ctl, llk_dev, (int)h->probs.size());
    const bool graph = !(flags & PTX_NO_GRAPH) && !h->profiling;
    const uint32_t base = flags & (PTX_UPDATE_OBJ | PTX_UPDATE_PROBE | PTX_NO_NORMALISE | PTX_UPDATE_BACKGROUND | forms);
    for (int c = 0; c < ncycles; ++c) {
        uint32_t f = base;
        if (c == 0 && (flags & PTX_DM_INIT_PSI)) f |= PTX_DM_INIT_PSI;
        if (graph) {
            cudaGraphExec_t ex;
            if ((st = get_graph(h, algos, f, &ex)) != PTX_OK) return st;
            cudaError_t e = cudaGraphLaunch(ex, s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        } else {
            if ((st = enqueue_cycle(h, algos, f, s)) != PTX_OK) return st;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "cycle launch");
    return PTX_OK;
}

}  // namespace

extern "C" {

ptx_status ptx_workspace_bytes(const ptx_problem* probs, int32_t nprob, size_t* scratch_bytes) {
    if (!probs || nprob < 1 || !scratch_bytes) return fail(PTX_ERR_INVALID_ARG, "null argument or nprob < 1");
    std::vector<ProbHost> v(nprob);
    for (int i = 0; i < nprob; ++i) {
        ptx_status st = check_problem(probs[i], i);
        if (st != PTX_OK) return st;
        v[i].p = probs[i];
        build_tiles(v[i], probs[i].positions);
    }
    size_t so, co, tot;
    compute_layout(v, &so, &co, &tot);
    *scratch_bytes = tot;
    return PTX_OK;
}

ptx_status ptx_create(ptx_handle** out, const ptx_problem* probs, int32_t nprob, void* scratch, size_t scratch_bytes,
                      void* stream) {
    if (!out) return fail(PTX_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!probs || nprob < 1) return fail(PTX_ERR_INVALID_ARG, "no problems");
    if (!scratch) return fail(PTX_ERR_INVALID_ARG, "scratch is null");
    if ((uintptr_t)scratch % kAlign) return fail(PTX_ERR_INVALID_ARG, "scratch must be %zu-byte aligned", kAlign);
    std::vector<ProbHost> v(nprob);
    for (int i = 0; i < nprob; ++i) {
        ptx_status st = check_problem(probs[i], i);
        if (st != PTX_OK) return st;
        v[i].p = probs[i];
        build_tiles(v[i], probs[i].positions);
    }
    size_t spec_off, ctl_off, total;
    size_t pers_off = 0;
    compute_layout(v, &spec_off, &ctl_off, &total, &pers_off);
    if (scratch_bytes < total)
        return fail(PTX_ERR_NOT_READY, "scratch of %zu bytes is smaller than the %zu needed", scratch_bytes, total);
    cudaError_t e = ensure_attributes();
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    ptx_handle* h = new ptx_handle();
    h->probs = std::move(v);
    h->scratch = (char*)scratch;
    h->scratch_bytes = scratch_bytes;
    h->spec_off = spec_off;
    h->ctl_off = ctl_off;
    h->pers_off = pers_off;
    h->spec_bytes = total - spec_off;
    h->ctl = (Ctl*)(h->scratch + ctl_off);
    cudaGetDevice(&h->device);
    if (cudaHostAlloc((void**)&h->err_host, sizeof(int), cudaHostAllocMapped) == cudaSuccess) {
        *h->err_host = 0;
        if (cudaHostGetDevicePointer((void**)&h->err_dev, h->err_host, 0) != cudaSuccess) h->err_dev = nullptr;
    } else {
        h->err_host = nullptr;
    }
    cudaGetLastError();
    for (ProbHost& ph : h->probs) {
        const KernelSet* ks = kernel_set(ph.p.N);
        const uint32_t C = (uint32_t)ks->reg_lines, N = (uint32_t)ph.p.N;
        const uint32_t th = (uint32_t)ph.tile_h;
        ph.tma_gather = ph.p.psi && N >= 64 && kObjTileW == 32 &&
                        encode_3d(&ph.tm_psi3, ph.p.psi, N, N, (uint64_t)ph.p.J * ph.p.K, 34, th) &&
                        encode_3d(&ph.tm_probe3, ph.p.probe, N, N, (uint64_t)ph.p.K, 34, th);
        ph.tma_io = ph.p.K == 1 && ks->col_tma && ks->col_tma_grid() > 0 &&
                    encode_2d(&ph.tm_io, 4, ph.p.iobs, N, (uint64_t)ph.p.J * N, C, N) &&
                    encode_2d(&ph.tm_mask, 1, h->scratch + ph.lay.mask, N, N, C, N);
    }
    cudaStream_t s = (cudaStream_t)stream;
    // zero everything the library owns, then copy positions and mask
    std::vector<std::vector<uint32_t>> mbits_host(h->probs.size());
    std::vector<std::vector<float>> nf_host(h->probs.size());
    e = cudaMemsetAsync(h->scratch, 0, spec_off, s);
    for (size_t i = 0; e == cudaSuccess && i < h->probs.size(); ++i) {
        ProbHost& ph = h->probs[i];
        // positions: the (row, col) int32 pairs are already laid out as int2
        std::vector<int32_t> pos(ph.p.positions, ph.p.positions + 2 * (size_t)ph.p.J);
        e = cudaMemcpyAsync(h->scratch + ph.lay.pos, pos.data(), pos.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        if (ph.p.mask) {
            e = cudaMemcpyAsync(h->scratch + ph.lay.mask, ph.p.mask, (size_t)ph.p.N * ph.p.N, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) break;
            if (use_reg_kernels(ph.ks, ph.p.K)) {
                mbits_host[i] = mask_bits(ph.ks, ph.p.N, ph.p.mask);
                e = cudaMemcpyAsync(h->scratch + ph.lay.mbits, mbits_host[i].data(), sizeof(uint32_t) * mbits_host[i].size(),
                                    cudaMemcpyHostToDevice, s);
                if (e != cudaSuccess) break;
            }
        }
        if (ph.p.nearfield > 0.0) {
            // t[k] = exp(-i pi c k^2 / N^2), k signed, in FP64 then rounded: h[ky][kx] = t[ky] t[kx]
            const int N = ph.p.N;
            nf_host[i].resize(2 * (size_t)N);
            for (int k = 0; k < N; ++k) {
                const double ks = k < (N + 1) / 2 ? k : k - N;
                const double ph_ = -M_PI * ph.p.nearfield * ks * ks / ((double)N * N);
                nf_host[i][2 * k] = (float)std::cos(ph_);
                nf_host[i][2 * k + 1] = (float)std::sin(ph_);
            }
            e = cudaMemcpyAsync(h->scratch + ph.lay.nf_t, nf_host[i].data(), sizeof(float) * nf_host[i].size(),
                                cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) break;
        }
        const std::vector<int>* lists[3] = {&ph.tile_ids, &ph.tile_ptr, &ph.tile_frames};
        const size_t offs[3] = {ph.lay.tile_ids, ph.lay.tile_ptr, ph.lay.tile_frames};
        for (int q = 0; q < 3 && e == cudaSuccess; ++q)
            if (!lists[q]->empty())
                e = cudaMemcpyAsync(h->scratch + offs[q], lists[q]->data(), sizeof(int) * lists[q]->size(),
                                    cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        ph.p.positions = nullptr;  // borrowed host arrays are not kept
        ph.p.mask = nullptr;
        fill_args(h, ph);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host staging vectors die here
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "ptx_create copy");
    }
    *out = h;
    return PTX_OK;
}

ptx_status ptx_ap_cycles(ptx_handle* h, int32_t ncycles, uint32_t flags, double* llk_dev, void* stream) {
    if (!h) return fail(PTX_ERR_INVALID_ARG, "null handle");
    if (flags & PTX_DM_INIT_PSI) return fail(PTX_ERR_INVALID_ARG, "PTX_DM_INIT_PSI is a DM flag");
    return run_cycles(h, std::vector<int>(h->probs.size(), ALGO_AP), ncycles, flags, llk_dev, stream);
}

ptx_status ptx_dm_cycles(ptx_handle* h, int32_t ncycles, uint32_t flags, double* llk_dev, void* stream) {
    if (!h) return fail(PTX_ERR_INVALID_ARG, "null handle");
    return run_cycles(h, std::vector<int>(h->probs.size(), ALGO_DM), ncycles, flags, llk_dev, stream);
}

ptx_status ptx_cycle_kernels(ptx_handle* h, int32_t algorithm, uint32_t flags, int64_t* count) {
    if (!h || !count) return fail(PTX_ERR_INVALID_ARG, "null handle or count");
    if (algorithm != ALGO_AP && algorithm != ALGO_DM) return fail(PTX_ERR_INVALID_ARG, "algorithm %d", algorithm);
    ptx_status st = check_device(h);
    if (st != PTX_OK) return st;
    const uint32_t f = flags & (PTX_UPDATE_OBJ | PTX_UPDATE_PROBE | PTX_NO_NORMALISE | PTX_UPDATE_BACKGROUND |
                                PTX_DM_INIT_PSI | PTX_FORM_TF32X2 | PTX_FORM_BF16X3 | PTX_FORM_BF16X2);
    const std::vector<int> algos(h->probs.size(), algorithm);
    if (h->persistent && h->pers_dirty && pers_eligible(h)) pers_build(h);  // sizes only; uploaded by the next cycle call
    cudaGraphExec_t ex;
    if ((st = get_graph(h, algos, f, &ex)) != PTX_OK) return st;
    GraphKey key{algos, f, h->lanes, h->tma | (h->tma_gather << 1) | (h->tc << 2)};
    auto it = h->graph_kernels.find(key);
    *count = it == h->graph_kernels.end() ? 0 : it->second;
    return PTX_OK;
}

ptx_status ptx_cycles(ptx_handle* h, int32_t ncycles, uint32_t flags, const int32_t* algorithms, double* llk_dev,
                      void* stream) {
    if (!h || !algorithms) return fail(PTX_ERR_INVALID_ARG, "null handle or algorithms");
    return run_cycles(h, std::vector<int>(algorithms, algorithms + h->probs.size()), ncycles, flags, llk_dev, stream);
}

ptx_status ptx_llk(ptx_handle* h, double* llk_dev, void* stream) {
    if (!h || !llk_dev) return fail(PTX_ERR_INVALID_ARG, "null handle or llk_dev");
    ptx_status st = check_device(h);
    if (st != PTX_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    for (size_t pi = 0; pi < h->probs.size(); ++pi) {
        ProbHost& ph = h->probs[pi];
        const bool pdl = pass_pdl(h, ph);
        for (int j0 = 0; j0 < ph.p.J; j0 += ph.B) {
            const int nb = std::min(ph.B, ph.p.J - j0);
            ph.ks->row_fwd(ph.args, j0, nb, X_PHI, s, pdl && j0 > 0);
            if (ph.p.nearfield > 0.0) {
                ph.ks->col_nf(ph.args, nb, +1, s);
                ph.ks->row_proj(ph.args, j0, nb, 1, s);
            } else {
                ph.ks->col(ph.args, j0, nb, COL_LLK, s, pdl);
            }
        }
        k_llk_reduce<<<1, 1024, 0, s>>>(ph.args, ph.p.N / ph.C2, llk_dev + pi);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ptx_llk launch");
    return PTX_OK;
}

ptx_status ptx_ml_grad(ptx_handle* h, void* grad_obj, void* grad_probe, double* llk_dev, void* stream) {
    if (!h) return fail(PTX_ERR_INVALID_ARG, "null handle");
    if (h->probs.size() != 1) return fail(PTX_ERR_INVALID_ARG, "ptx_ml_grad needs a single-problem handle");
    ptx_status st = check_device(h);
    if (st != PTX_OK) return st;
    for (const ProbHost& q : h->probs)
        if (q.p.nearfield > 0.0) return fail(PTX_ERR_UNSUPPORTED, "%s: the near field serves AP, DM and the LLK only", "ptx_ml_grad");
    cudaStream_t s = (cudaStream_t)stream;
    ProbHost& ph = h->probs[0];
    ProbArgs a = ph.args;
    a.grad_obj = (float2*)grad_obj;
    a.grad_probe = (float2*)grad_probe;
    cudaError_t e = cudaSuccess;
    if (grad_obj) e = cudaMemsetAsync(grad_obj, 0, sizeof(float2) * (size_t)a.Ho * a.Wo, s);
    if (e == cudaSuccess && grad_probe) e = cudaMemsetAsync(grad_probe, 0, sizeof(float2) * (size_t)a.K * a.N * a.N, s);
    if (e != cudaSuccess) return cuda_fail(e, "ptx_ml_grad memset");
    const bool pdl = pass_pdl(h, ph);
    for (int j0 = 0; j0 < ph.p.J; j0 += ph.B) {
        const int nb = std::min(ph.B, ph.p.J - j0);
        ph.ks->row_fwd(a, j0, nb, X_PHI, s, pdl && j0 > 0);
        ph.ks->col(a, j0, nb, COL_GRAD, s, pdl);
        if (grad_obj || grad_probe)
            ph.ks->row_bwd(a, j0, nb, std::min(ph.G3, nb), BWD_GRAD, grad_obj != nullptr, grad_probe != nullptr, s,
                           pdl);
    }
    if (llk_dev) k_llk_reduce<<<1, 1024, 0, s>>>(a, a.N / a.C2, llk_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ptx_ml_grad launch");
    return PTX_OK;
}

namespace {

CgArgs cg_args(ptx_handle* h, ProbHost& ph) {
    CgArgs c;
    const size_t no = (size_t)ph.p.Ho * ph.p.Wo, npr = (size_t)ph.p.K * ph.p.N * ph.p.N;
    float2* o = (float2*)(h->scratch + ph.lay.cg_obj);
    float2* pr = (float2*)(h->scratch + ph.lay.cg_probe);
    c.g_obj = o;
    c.gp_obj = o + no;
    c.d_obj = o + 2 * no;
    c.g_probe = pr;
    c.gp_probe = pr + npr;
    c.d_probe = pr + 2 * npr;
    c.n_obj = no;
    c.n_probe = npr;
    c.cg = (double*)(h->scratch + ph.lay.cg);
    c.cg_part = c.cg + 8;
    return c;
}

// Line-search pass: L'(0), L''(0) along (dir_obj, dir_probe) into out[0..1].
ptx_status enqueue_line_coeffs(ptx_handle* h, ProbHost& ph, const float2* d_obj, const float2* d_probe, double* out,
                               cudaStream_t s) {
    ProbArgs a = ph.args;
    a.dir_obj = d_obj;
    a.dir_probe = d_probe;
    // work stack per frame: the waves A, B (and C with both parts of the
    // direction) of one mode for the register kernels, 3 K waves otherwise
    const int waves = (ph.p.K == 1 && ph.ks->reg_lines > 0) ? ((d_obj && d_probe) ? 3 : 2) : 3 * ph.p.K;
    const size_t frame_w = (size_t)waves * ph.p.N * ph.p.N * sizeof(float2);
    size_t B = h->spec_bytes / frame_w;
    if (B < 1) B = 1;
    if (B > (size_t)ph.p.J) B = ph.p.J;
    if (B > 32768) B = 32768;
    const bool pdl = pass_pdl(h, ph);
    for (int j0 = 0; j0 < ph.p.J; j0 += (int)B) {
        const int nb = std::min((int)B, ph.p.J - j0);
        ph.ks->row_fwd_ls(a, j0, nb, pdl && j0 > 0, s);
        ph.ks->col_ls(a, j0, nb, pdl, s);
    }
    // partial pairs per frame: one per column block of the line-search column pass
    k_ls_reduce<<<1, 1024, 0, s>>>(a.ls_part, (size_t)ph.p.J * (ph.p.N / ls_cols(ph.ks, ph.p.K)), out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "line-search launch");
    return PTX_OK;
}

// Gradient of the LLK into (g_obj, g_probe) (each may be null), LLK into llk_out.
ptx_status enqueue_grad(ptx_handle* h, ProbHost& ph, float2* g_obj, float2* g_probe, double* llk_out, cudaStream_t s) {
    ProbArgs a = ph.args;
    a.grad_obj = g_obj;
    a.grad_probe = g_probe;
    cudaError_t e = cudaSuccess;
    if (g_obj) e = cudaMemsetAsync(g_obj, 0, sizeof(float2) * (size_t)a.Ho * a.Wo, s);
    if (e == cudaSuccess && g_probe) e = cudaMemsetAsync(g_probe, 0, sizeof(float2) * (size_t)a.K * a.N * a.N, s);
    if (e != cudaSuccess) return cuda_fail(e, "gradient memset");
    set_batch(ph, h->spec_bytes, 1, h->batch_cap, h->bwd_slots);
    const bool pdl = pass_pdl(h, ph);
    for (int j0 = 0; j0 < ph.p.J; j0 += ph.B) {
        const int nb = std::min(ph.B, ph.p.J - j0);
        ph.ks->row_fwd(a, j0, nb, X_PHI, s, pdl && j0 > 0);
        ph.ks->col(a, j0, nb, COL_GRAD, s, pdl);
        if (g_obj || g_probe)
            ph.ks->row_bwd(a, j0, nb, std::min(ph.G3, nb), BWD_GRAD, g_obj != nullptr, g_probe != nullptr, s, pdl);
    }
    if (llk_out) k_llk_reduce<<<1, 1024, 0, s>>>(a, a.N / a.C2, llk_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gradient launch");
    return PTX_OK;
}

}  // namespace

ptx_status ptx_ml_line_coeffs(ptx_handle* h, const void* d_obj, const void* d_probe, double* coeffs_dev,
                              void* stream) {
    if (!h || !coeffs_dev) return fail(PTX_ERR_INVALID_ARG, "null handle or coeffs_dev");
    if (h->probs.size() != 1) return fail(PTX_ERR_INVALID_ARG, "ML needs a single-problem handle");
    ptx_status st = check_device(h);
    if (st != PTX_OK) return st;
    for (const ProbHost& q : h->probs)
        if (q.p.nearfield > 0.0) return fail(PTX_ERR_UNSUPPORTED, "%s: the near field serves AP, DM and the LLK only", "ptx_ml_line_coeffs");
    return enqueue_line_coeffs(h, h->probs[0], (const float2*)d_obj, (const float2*)d_probe, coeffs_dev,
                               (cudaStream_t)stream);
}

ptx_status ptx_ml_cycles(ptx_handle* h, int32_t ncycles, uint32_t flags, double* llk_dev, void* stream) {
    if (!h) return fail(PTX_ERR_INVALID_ARG, "null handle");
    if (h->probs.size() != 1) return fail(PTX_ERR_INVALID_ARG, "ML needs a single-problem handle");
    if (ncycles < 0) return fail(PTX_ERR_INVALID_ARG, "ncycles=%d must be >= 0", ncycles);
    const uint32_t known = PTX_UPDATE_OBJ | PTX_UPDATE_PROBE | PTX_ML_RESTART;
    if (flags & ~known) return fail(PTX_ERR_INVALID_ARG, "unknown flag bits 0x%x", flags & ~known);
    ptx_status st = check_device(h);
    if (st != PTX_OK) return st;
    for (const ProbHost& q : h->probs)
        if (q.p.nearfield > 0.0) return fail(PTX_ERR_UNSUPPORTED, "%s: the near field serves AP, DM and the LLK only", "ptx_ml_cycles");
    cudaStream_t s = (cudaStream_t)stream;
    ProbHost& ph = h->probs[0];
    CgArgs c = cg_args(h, ph);
    const bool uo = flags & PTX_UPDATE_OBJ, up = flags & PTX_UPDATE_PROBE;
    cudaError_t e = cudaSuccess;
    if (flags & PTX_ML_RESTART) {
        e = cudaMemsetAsync(c.gp_obj, 0, 2 * sizeof(float2) * c.n_obj, s);  // previous gradient and direction
        if (e == cudaSuccess) e = cudaMemsetAsync(c.gp_probe, 0, 2 * sizeof(float2) * c.n_probe, s);
        if (e != cudaSuccess) return cuda_fail(e, "ML restart memset");
    }
    const int nblk = kCgBlocks;
    for (int cyc = 0; cyc < ncycles; ++cyc) {
        // gradient (zero where a part is not updated) and the LLK before the step
        if (!uo && (e = cudaMemsetAsync(c.g_obj, 0, sizeof(float2) * c.n_obj, s)) != cudaSuccess)
            return cuda_fail(e, "memset");
        if (!up && (e = cudaMemsetAsync(c.g_probe, 0, sizeof(float2) * c.n_probe, s)) != cudaSuccess)
            return cuda_fail(e, "memset");
        if ((st = enqueue_grad(h, ph, uo ? c.g_obj : nullptr, up ? c.g_probe : nullptr, llk_dev ? llk_dev + cyc : nullptr,
                               s)) != PTX_OK)
            return st;
        if ((e = cudaMemsetAsync(c.cg, 0, 8 * sizeof(double), s)) != cudaSuccess) return cuda_fail(e, "memset");
        k_cg_dots<<<nblk, 256, 0, s>>>(c);
        k_cg_reduce<<<1, 256, 0, s>>>(c);
        k_cg_direction<<<nblk, 256, 0, s>>>(c);
        if ((st = enqueue_line_coeffs(h, ph, uo ? c.d_obj : nullptr, up ? c.d_probe : nullptr, c.cg + 3, s)) != PTX_OK)
            return st;
        k_cg_step<<<nblk, 256, 0, s>>>(c, ph.args.obj, ph.args.probe);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ML cycle launch");
    return PTX_OK;
}

ptx_status ptx_normalise(ptx_handle* h, uint32_t flags, void* stream) {
    if (!h) return fail(PTX_ERR_INVALID_ARG, "null handle");
    const uint32_t known = PTX_UPDATE_OBJ | PTX_UPDATE_PROBE | PTX_STAGE_PROBE | PTX_STAGE_OBJ_GATHER |
                           PTX_STAGE_OBJ_NORMALISE;
    if (flags & ~known) return fail(PTX_ERR_INVALID_ARG, "unknown flag bits 0x%x", flags & ~known);
    ptx_status st = check_device(h);
    if (st != PTX_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int stages = (int)(flags & (PTX_STAGE_PROBE | PTX_STAGE_OBJ_GATHER | PTX_STAGE_OBJ_NORMALISE));
    if (flags & PTX_UPDATE_PROBE) stages |= STAGE_PROBE;
    if (flags & PTX_UPDATE_OBJ) stages |= STAGE_OBJ_GATHER | STAGE_OBJ_NORMALISE;
    for (auto& ph : h->probs) {
        enqueue_stages(h, ph, stages, s);
        cudaError_t e = cudaMemsetAsync(ph.args.maxbits, 0, 2 * sizeof(unsigned), s);
        if (e != cudaSuccess) return cuda_fail(e, "ptx_normalise memset");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ptx_normalise launch");
    return PTX_OK;
}

ptx_status ptx_accumulators(ptx_handle* h, int32_t p, void** obj_acc, size_t* obj_acc_bytes, void** probe_acc,
                            size_t* probe_acc_bytes) {
    if (!h || p < 0 || p >= (int)h->probs.size()) return fail(PTX_ERR_INVALID_ARG, "bad handle or problem index");
    const ProbHost& ph = h->probs[p];
    if (obj_acc) *obj_acc = ph.args.acc_obj;
    if (obj_acc_bytes) *obj_acc_bytes = sizeof(float4) * (size_t)ph.p.Ho * ph.p.Wo;
    if (probe_acc) *probe_acc = ph.args.acc_probe;
    if (probe_acc_bytes) *probe_acc_bytes = sizeof(float4) * (size_t)ph.p.K * ph.p.N * ph.p.N;
    return PTX_OK;
}

ptx_status ptx_set_param(ptx_handle* h, const char* name, double value) {
    if (!h || !name) return fail(PTX_ERR_INVALID_ARG, "null handle or name");
    if (!(value >= 0.0) || !std::isfinite(value)) return fail(PTX_ERR_INVALID_ARG, "%s must be finite and >= 0", name);
    if (!strcmp(name, "alpha_obj")) {
        h->alpha_obj = value;
    } else if (!strcmp(name, "alpha_probe")) {
        h->alpha_probe = value;
    } else if (!strcmp(name, "lanes")) {
        if (value < 1 || value > kMaxLanes || value != (int)value)
            return fail(PTX_ERR_INVALID_ARG, "lanes must be an integer in 1..%d", kMaxLanes);
        h->lanes = (int)value;
    } else if (!strcmp(name, "tma")) {
        if (value != 0.0 && value != 1.0) return fail(PTX_ERR_INVALID_ARG, "tma must be 0 or 1");
        h->tma = (int)value;
    } else if (!strcmp(name, "tc")) {
        if (value != 0.0 && value != 1.0 && value != 2.0 && value != 3.0)
            return fail(PTX_ERR_INVALID_ARG, "tc must be 0 (FP32), 1 (TF32X2), 2 (BF16X3) or 3 (BF16X2)");
        h->tc = (int)value;
    } else if (!strcmp(name, "tma_gather")) {
        if (value != 0.0 && value != 1.0) return fail(PTX_ERR_INVALID_ARG, "tma_gather must be 0 or 1");
        h->tma_gather = (int)value;
    } else if (!strcmp(name, "bwd_slots")) {
        if (value != (int)value || value < 0 || value > 4096)
            return fail(PTX_ERR_INVALID_ARG, "bwd_slots must be an integer in 0..4096");
        h->bwd_slots = (int)value;
    } else if (!strcmp(name, "persistent")) {
        if (value != 0.0 && value != 1.0) return fail(PTX_ERR_INVALID_ARG, "persistent must be 0 or 1");
        h->persistent = (int)value;
    } else if (!strcmp(name, "persistent_selftest")) {
        if (value != 0.0 && value != 1.0) return fail(PTX_ERR_INVALID_ARG, "persistent_selftest must be 0 or 1");
        h->pers_selftest = (int)value;
    } else if (!strcmp(name, "tc_rows")) {
        if (value != 0.0 && value != 1.0) return fail(PTX_ERR_INVALID_ARG, "tc_rows must be 0 or 1");
        h->tc_rows = (int)value;
    } else if (!strcmp(name, "tc_selftest")) {
        if (value != 0.0 && value != 1.0) return fail(PTX_ERR_INVALID_ARG, "tc_selftest must be 0 or 1");
        h->tc_selftest = (int)value;
    } else if (!strcmp(name, "pdl")) {
        if (value != 0.0 && value != 1.0) return fail(PTX_ERR_INVALID_ARG, "pdl must be 0 or 1");
        h->pdl = (int)value;
    } else if (!strcmp(name, "batch_frames")) {
        if (value != (int)value || value > 32768)
            return fail(PTX_ERR_INVALID_ARG, "batch_frames must be an integer in 0..32768");
        h->batch_cap = (int)value;
    } else {
        return fail(PTX_ERR_INVALID_ARG, "unknown parameter '%s'", name);
    }
    drop_graphs(h);  // the captured graphs hold the old value
    h->pers_dirty = true;
    return PTX_OK;
}

ptx_status ptx_fft2(void* data, int32_t nframes, int32_t N, int32_t direction, void* stream) {
    if (!data || nframes < 0) return fail(PTX_ERR_INVALID_ARG, "null data or negative nframes");
    if (direction != -1 && direction != 1) return fail(PTX_ERR_INVALID_ARG, "direction must be -1 or +1");
    if (!supported_N(N)) return fail(PTX_ERR_UNSUPPORTED, "frame size N=%d is not supported", N);
    if (nframes == 0) return PTX_OK;
    if (nframes > 65535) return fail(PTX_ERR_INVALID_ARG, "nframes=%d exceeds 65535 per call", nframes);
    cudaError_t e = ensure_attributes();
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    kernel_set(N)->fft2((float2*)data, nframes, direction, (cudaStream_t)stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ptx_fft2 launch");
    return PTX_OK;
}

ptx_status ptx_counts_to_float(float* dst, const uint16_t* src, size_t n, void* stream) {
    if (n == 0) return PTX_OK;
    if (!dst || !src) return fail(PTX_ERR_INVALID_ARG, "null dst or src");
    if ((uintptr_t)dst % 16 || (uintptr_t)src % 16) return fail(PTX_ERR_INVALID_ARG, "dst and src must be 16-byte aligned");
    k_counts_to_float<<<4 * 152, 256, 0, (cudaStream_t)stream>>>(src, dst, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ptx_counts_to_float launch");
    return PTX_OK;
}

ptx_status ptx_encode_counts8(const uint16_t* src, size_t n, uint8_t* out8, uint32_t* esc_index,
                              uint16_t* esc_value, size_t cap, size_t* n_esc) {
    if (!n_esc) return fail(PTX_ERR_INVALID_ARG, "n_esc is null");
    *n_esc = 0;
    if (n >= ((size_t)1 << 32)) return fail(PTX_ERR_INVALID_ARG, "n must be below 2^32");
    if (n == 0) return PTX_OK;
    const bool count_only = cap == 0 && !out8 && !esc_index && !esc_value;
    if (!src || (!count_only && (!out8 || (cap > 0 && (!esc_index || !esc_value)))))
        return fail(PTX_ERR_INVALID_ARG, "null array");
    size_t k = 0;
    for (size_t i = 0; i < n; ++i) {
        const uint16_t c = src[i];
        if (!count_only) out8[i] = c < 255 ? (uint8_t)c : (uint8_t)255;
        if (c >= 255) {
            if (!count_only && k < cap) {
                esc_index[k] = (uint32_t)i;
                esc_value[k] = c;
            }
            ++k;
        }
    }
    *n_esc = k;
    if (!count_only && k > cap) return fail(PTX_ERR_OUT_OF_BOUNDS, "%zu escapes exceed the capacity %zu", k, cap);
    return PTX_OK;
}

ptx_status ptx_counts8_to_float(float* dst, const uint8_t* src8, size_t n, const uint32_t* esc_index,
                                const uint16_t* esc_value, size_t n_esc, void* stream) {
    if (n == 0) return PTX_OK;
    if (!dst || !src8) return fail(PTX_ERR_INVALID_ARG, "null dst or src8");
    if (n >= ((size_t)1 << 32)) return fail(PTX_ERR_INVALID_ARG, "n must be below 2^32");
    if ((uintptr_t)dst % 16 || (uintptr_t)src8 % 16)
        return fail(PTX_ERR_INVALID_ARG, "dst and src8 must be 16-byte aligned");
    if (n_esc > 0 && (!esc_index || !esc_value)) return fail(PTX_ERR_INVALID_ARG, "null escape arrays");
    cudaStream_t s = (cudaStream_t)stream;
    k_counts8_to_float<<<4 * 152, 256, 0, s>>>(src8, dst, n);
    if (n_esc > 0) {
        const int blocks = (int)std::min<size_t>((n_esc + 255) / 256, 4 * 152);
        k_counts8_escapes<<<blocks, 256, 0, s>>>(esc_index, esc_value, dst, n_esc, n);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ptx_counts8_to_float launch");
    return PTX_OK;
}

ptx_status ptx_fma_peak(int32_t blocks, int32_t iters, float* sink, double* flops, void* stream) {
    if (blocks < 1 || iters < 1 || !sink || !flops)
        return fail(PTX_ERR_INVALID_ARG, "blocks and iters must be >= 1, sink and flops non-null");
    *flops = 32.0 * 256.0 * (double)blocks * (double)iters;
    k_fma_peak<<<blocks, 256, 0, (cudaStream_t)stream>>>(sink, iters, 0.999999f, 1e-6f);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ptx_fma_peak launch");
    return PTX_OK;
}

ptx_status ptx_accumulate_shifts(int32_t J, const float* shifts, double step, double max_shift, int32_t max_row,
                                 int32_t max_col, double* pos_subpixel, int32_t* positions, int32_t* moved) {
    if (J < 0 || !moved || (J > 0 && (!shifts || !pos_subpixel || !positions)))
        return fail(PTX_ERR_INVALID_ARG, "J >= 0 and non-null arrays needed");
    if (!(max_shift >= 0.0) || max_row < 0 || max_col < 0)
        return fail(PTX_ERR_INVALID_ARG, "max_shift, max_row and max_col must be >= 0");
    const double hi[2] = {(double)max_row, (double)max_col};
    int32_t n = 0;
    for (int32_t j = 0; j < J; ++j) {
        bool changed = false;
        for (int a = 0; a < 2; ++a) {
            const double d = std::min(std::max(step * (double)shifts[2 * j + a], -max_shift), max_shift);
            const double v = std::min(std::max(pos_subpixel[2 * j + a] + d, 0.0), hi[a]);
            pos_subpixel[2 * j + a] = v;
            const int32_t r = (int32_t)std::nearbyint(v);  // round half to even (default rounding mode)
            changed |= r != positions[2 * j + a];
            positions[2 * j + a] = r;
        }
        n += changed ? 1 : 0;
    }
    *moved = n;
    return PTX_OK;
}

ptx_status ptx_profile_enable(ptx_handle* h, int32_t enable) {
    if (!h) return fail(PTX_ERR_INVALID_ARG, "null handle");
    h->profiling = enable != 0;
    h->ev_used.clear();
    return PTX_OK;
}

ptx_status ptx_profile_read(ptx_handle* h, int32_t nkinds, int64_t* launches, double* total_ms) {
    if (!h || nkinds < 0 || (nkinds > 0 && (!launches || !total_ms)))
        return fail(PTX_ERR_INVALID_ARG, "null handle or output arrays");
    for (int k = 0; k < nkinds; ++k) {
        launches[k] = 0;
        total_ms[k] = 0.0;
    }
    for (const auto& u : h->ev_used) {
        cudaError_t e = cudaEventSynchronize(h->ev_pool[u.second + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, h->ev_pool[u.second], h->ev_pool[u.second + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        if (u.first < nkinds) {
            launches[u.first] += 1;
            total_ms[u.first] += ms;
        }
    }
    return PTX_OK;
}

ptx_status ptx_position_shifts(ptx_handle* h, int32_t p, float filter_ratio, float* shifts, void* stream) {
    if (!h || !shifts) return fail(PTX_ERR_INVALID_ARG, "null handle or shifts");
    if (p < 0 || p >= (int)h->probs.size()) return fail(PTX_ERR_INVALID_ARG, "problem %d out of range", p);
    if (!(filter_ratio >= 0.f)) return fail(PTX_ERR_INVALID_ARG, "filter_ratio must be >= 0");
    ProbHost& ph = h->probs[p];
    if (!ph.p.psi) return fail(PTX_ERR_INVALID_ARG, "position shifts need the psi array of the last cycle");
    ptx_status st = check_device(h);
    if (st != PTX_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int bands = (ph.p.N + 7) / 8;
    double* part = (double*)(h->scratch + ph.lay.pos_part);
    k_pos_sums<<<dim3(bands, ph.p.J), 256, 0, s>>>(ph.args, part);
    k_pos_solve<<<1, 1024, 0, s>>>(part, ph.p.J, bands, filter_ratio, shifts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ptx_position_shifts launch");
    return PTX_OK;
}

ptx_status ptx_set_positions(ptx_handle* h, int32_t p, const int32_t* positions, void* stream) {
    if (!h || !positions) return fail(PTX_ERR_INVALID_ARG, "null handle or positions");
    if (p < 0 || p >= (int)h->probs.size()) return fail(PTX_ERR_INVALID_ARG, "problem %d out of range", p);
    ProbHost& ph = h->probs[p];
    for (int j = 0; j < ph.p.J; ++j) {
        const int r = positions[2 * j], c = positions[2 * j + 1];
        if (r < 0 || c < 0 || r > ph.p.Ho - ph.p.N || c > ph.p.Wo - ph.p.N)
            return fail(PTX_ERR_OUT_OF_BOUNDS, "position %d = (%d, %d) puts the %dx%d patch outside the %dx%d object", j,
                        r, c, ph.p.N, ph.p.N, ph.p.Ho, ph.p.Wo);
    }
    ptx_status st = check_device(h);
    if (st != PTX_OK) return st;
    build_tiles(ph, positions);
    fill_args(h, ph);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h->scratch + ph.lay.pos, positions, sizeof(int32_t) * 2 * (size_t)ph.p.J,
                                    cudaMemcpyHostToDevice, s);
    const std::vector<int>* lists[3] = {&ph.tile_ids, &ph.tile_ptr, &ph.tile_frames};
    const size_t offs[3] = {ph.lay.tile_ids, ph.lay.tile_ptr, ph.lay.tile_frames};
    for (int q = 0; q < 3 && e == cudaSuccess; ++q)
        if (!lists[q]->empty())
            e = cudaMemcpyAsync(h->scratch + offs[q], lists[q]->data(), sizeof(int) * lists[q]->size(),
                                cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host arrays are not kept
    if (e != cudaSuccess) return cuda_fail(e, "ptx_set_positions copy");
    drop_graphs(h);  // captured cycles hold the old tile count
    return PTX_OK;
}

const char* ptx_last_error(void) { return g_last_error.c_str(); }

ptx_status ptx_wait_selftest(ptx_handle* h, int32_t limit_us, void* stream) {
    if (!h) return fail(PTX_ERR_INVALID_ARG, "null handle");
    if (limit_us < 1 || limit_us > 1000000) return fail(PTX_ERR_INVALID_ARG, "limit_us=%d must be in 1..1000000", limit_us);
    ptx_status st = check_device(h);
    if (st != PTX_OK) return st;
    if (!h->err_dev) return fail(PTX_ERR_NOT_READY, "the handle has no device error flag");
    k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(h->err_dev, 1000ull * (unsigned long long)limit_us);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "self-test launch");
    return PTX_OK;
}

void ptx_destroy(ptx_handle* h) {
    if (!h) return;
    drop_graphs(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    for (int l = 0; l < kMaxLanes; ++l) {
        if (h->lane_stream[l]) cudaStreamDestroy(h->lane_stream[l]);
        if (h->join_ev[l]) cudaEventDestroy(h->join_ev[l]);
    }
    for (cudaEvent_t e : h->prob_ev) cudaEventDestroy(e);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->err_host) cudaFreeHost(h->err_host);
    delete h;
}

}  // extern "C"
