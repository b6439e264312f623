// ptx_llk_static: the Poisson log-likelihood of ptx_llk for callers that cannot
// allocate device memory, with all working memory in one fixed device array.
//
// Who needs it: code that runs where cudaMalloc (or any allocating library
// routine, torch's caching allocator included) is not available or not
// allowed — e.g. a plug-in called from a host application that owns all
// device memory and hands out only its input and output buffers, or a
// real-time loop that must not enter the allocator.  Such callers pass their
// inputs (object, probe, intensities on the device; positions and mask on the
// host) and an output buffer, and this entry point uses nothing else.
//
// The working memory is the file-scope array g_llk_scratch below
// (kStaticScratchBytes = 16 MiB); every GPU that loads the library holds it
// until the process exits.  Host code cannot use the array's name as a device
// address, so every call looks the address up with cudaGetSymbolAddress (with
// the caller's device current; the lookup does not synchronise).  The first
// call that sees a given address on a device (the first call on the device, or
// the first after a cudaDeviceReset that reloaded the module) also clears the
// mask region of the array and sets the kernels' attributes; that call
// synchronises the device once and must therefore come before any stream
// capture.  All calls share the
// array and it keeps the last call's contents: each call rewrites every byte
// it reads (positions, mask, Fourier work stack, partial sums) before reading
// it, so calls that run one after the other are independent, but calls that
// overlap on the GPU (different streams or devices' threads racing on one
// device) race on the array and give undefined results.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <vector>

#include "../../include/ptycho.h"
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set(int N);
void set_last_error(const char* msg);
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
}  // namespace ptx

namespace {

constexpr size_t kStaticScratchBytes = PTX_STATIC_SCRATCH_BYTES;
// regions of the array
constexpr size_t kPosOff = 0;                         // int2 positions, up to kMaxFrames
constexpr size_t kMaxFrames = 65536;
constexpr size_t kMaskOff = kPosOff + kMaxFrames * 8;  // uint8 mask, up to 512 x 512
constexpr size_t kMaskBytes = 512 * 512;
constexpr size_t kPartOff = kMaskOff + kMaskBytes;    // double LLK partial sums
constexpr size_t kMaxParts = 65536;
constexpr size_t kSpecOff = kPartOff + kMaxParts * 8;  // Fourier work stack
static_assert(kSpecOff % 256 == 0, "regions are 256-byte aligned");
static_assert(kSpecOff < kStaticScratchBytes, "work stack region must exist");

__device__ __align__(256) unsigned char g_llk_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
void* g_ready[64] = {};  // per device ordinal: the address whose one-time set-up is done

ptx_status fail(ptx_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ptx::set_last_error(buf);
    return st;
}

// Every call: the array's device address on the current device.  The first
// call that sees that address: cleared mask region, kernel attributes.
ptx_status setup_device(int dev, unsigned char** out) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_llk_scratch);
    if (e != cudaSuccess) return fail(PTX_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_ready[dev] == ptr) {
        *out = (unsigned char*)ptr;
        return PTX_OK;
    }
    cudaError_t (*attrs[])() = {ptx::set_attrs_8,   ptx::set_attrs_12,  ptx::set_attrs_16,  ptx::set_attrs_32,
                                ptx::set_attrs_64,  ptx::set_attrs_128, ptx::set_attrs_192, ptx::set_attrs_256,
                                ptx::set_attrs_384, ptx::set_attrs_512, ptx::set_attrs_80,  ptx::set_attrs_160,
                                ptx::set_attrs_224, ptx::set_attrs_400, ptx::set_attrs_448};
    for (auto f : attrs)
        if ((e = f()) != cudaSuccess) return fail(PTX_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    if ((e = cudaMemset((char*)ptr + kMaskOff, 0, kMaskBytes)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess)
        return fail(PTX_ERR_CUDA, "clearing the static scratch: %s", cudaGetErrorString(e));
    g_ready[dev] = ptr;
    *out = (unsigned char*)ptr;
    return PTX_OK;
}

// columns per block of the column pass (= LLK partial sums per frame)
int lines_for(const ptx::KernelSet* ks, int N, int K) {
    if (ptx::use_reg_kernels(ks, K)) return ks->reg_cols;
    int L = 1;
    while (K * L * 2 <= ks->max_lines && N % (L * 2) == 0) L *= 2;
    return L;
}

}  // namespace

extern "C" ptx_status ptx_llk_static(int32_t N, int32_t K, int32_t J, int32_t Ho, int32_t Wo, const void* obj,
                                     const void* probe, const int32_t* positions, const float* iobs,
                                     const uint8_t* mask, double* llk_dev, void* stream) {
    static const int sizes[] = PTX_SUPPORTED_SIZES;
    bool ok_n = false;
    for (int s : sizes) ok_n |= (s == N);
    if (!ok_n) return fail(PTX_ERR_UNSUPPORTED, "frame size N=%d is not supported", N);
    if (K < 1 || K > PTX_MAX_MODES) return fail(PTX_ERR_UNSUPPORTED, "K=%d modes (1..%d)", K, PTX_MAX_MODES);
    if (J < 1 || Ho < N || Wo < N) return fail(PTX_ERR_INVALID_ARG, "J >= 1 and an object of at least N x N needed");
    if (!obj || !probe || !positions || !iobs || !llk_dev)
        return fail(PTX_ERR_INVALID_ARG, "obj, probe, positions, iobs and llk_dev must be non-null");
    if ((uintptr_t)iobs % 16 || (uintptr_t)probe % 16 || (uintptr_t)obj % 8)
        return fail(PTX_ERR_INVALID_ARG, "iobs and probe must be 16-byte aligned, obj 8-byte");
    const ptx::KernelSet* ks = ptx::kernel_set(N);
    const int L = lines_for(ks, N, K);
    const size_t nparts = (size_t)N / L;
    const size_t frame_bytes = (size_t)K * N * N * sizeof(float2);
    const size_t spec_bytes = kStaticScratchBytes - kSpecOff;
    if ((size_t)J > kMaxFrames)
        return fail(PTX_ERR_UNSUPPORTED, "J=%d exceeds the %zu frames of the static scratch", J, kMaxFrames);
    if ((size_t)J * nparts > kMaxParts)
        return fail(PTX_ERR_UNSUPPORTED, "J=%d frames of %dx%d need %zu partial sums, more than the %zu of the static scratch",
                    J, N, N, (size_t)J * nparts, kMaxParts);
    if (frame_bytes > spec_bytes)
        return fail(PTX_ERR_UNSUPPORTED, "one frame's work stack (%zu bytes for K=%d, N=%d) exceeds the %zu bytes of the static scratch",
                    frame_bytes, K, N, spec_bytes);
    for (int j = 0; j < J; ++j) {
        const int r = positions[2 * j], c = positions[2 * j + 1];
        if (r < 0 || c < 0 || r > Ho - N || c > Wo - N)
            return fail(PTX_ERR_OUT_OF_BOUNDS, "position %d = (%d, %d) puts the %dx%d patch outside the %dx%d object", j,
                        r, c, N, N, Ho, Wo);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PTX_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fail(PTX_ERR_UNSUPPORTED, "device ordinal %d", dev);
    unsigned char* base = nullptr;
    ptx_status st = setup_device(dev, &base);
    if (st != PTX_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // inputs that live in the array: positions and (a nonzero) mask; the mask
    // region is zero from set-up and is cleared again after a masked call
    e = cudaMemcpyAsync(base + kPosOff, positions, (size_t)J * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && mask) e = cudaMemcpyAsync(base + kMaskOff, mask, (size_t)N * N, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(PTX_ERR_CUDA, "copying positions / mask: %s", cudaGetErrorString(e));
    ptx::ProbArgs a{};
    a.N = N;
    a.K = K;
    a.J = J;
    a.Ho = Ho;
    a.Wo = Wo;
    a.obj = (float2*)obj;
    a.probe = (float2*)probe;
    a.iobs = iobs;
    a.pos = (const int2*)(base + kPosOff);
    a.mask = base + kMaskOff;
    a.spec = (float2*)(base + kSpecOff);
    a.llk_part = (double*)(base + kPartOff);
    a.L1 = a.C2 = a.L3 = L;
    size_t B = spec_bytes / frame_bytes;
    if (B > (size_t)J) B = J;
    if (B > 32768) B = 32768;
    for (int j0 = 0; j0 < J; j0 += (int)B) {
        const int nb = (int)std::min<size_t>(B, (size_t)(J - j0));
        ks->row_fwd(a, j0, nb, ptx::X_PHI, s, false);
        ks->col(a, j0, nb, ptx::COL_LLK, s, false);
    }
    ptx::k_llk_reduce<<<1, 1024, 0, s>>>(a, (int)nparts, llk_dev);
    if (mask) e = cudaMemsetAsync(base + kMaskOff, 0, (size_t)N * N, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PTX_ERR_CUDA, "ptx_llk_static launch: %s", cudaGetErrorString(e));
    return PTX_OK;
}
