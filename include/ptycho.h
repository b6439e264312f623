/*
 * libptycho - far-field ptychography projection cycle on one NVIDIA GB300 (sm_103a).
 *
 * The operations follow the ptychography operators of Favre-Nicolin et al.,
 * "PyNX: high performance computing toolkit for coherent X-ray imaging based on
 * operators" (2020): ObjProbe2Psi, FT / IFT, ApplyAmplitude, Psi2ObjProbe, AP,
 * DM, LLK and ML (appendix operator table; feature list of Section 4).
 *
 * Conventions for every entry point:
 *   - Complex arrays are complex64 (interleaved float re, im), C-contiguous.
 *   - A position (row, col) is the top-left corner of the frame's N x N object
 *     patch: the exit wave of frame j, mode k is Phi_jk(y, x) = P_k(y, x) O(row_j + y, col_j + x)
 *     (the paper's Psi_j(r) = O(r) P(r - r_j), Section 4 / operator table).
 *   - The 2D Fourier transform is orthonormal (forward and inverse both scaled
 *     by 1/N); intensities and the mask are in FFT order (zero frequency at [0][0]).
 *   - "device" pointers are CUDA global-memory pointers on the current device;
 *     "host" pointers are ordinary process memory.  The caller owns every array it
 *     passes; the library never frees caller memory.
 *   - A stream argument is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream: arguments are checked on
 *     the host before anything is enqueued, results are valid once the stream
 *     has reached the call.  No entry point except ptx_create allocates device
 *     memory, and none synchronises the host with the device after ptx_create.
 *   - Errors come back as a ptx_status; ptx_last_error() gives the text of the
 *     last failure on the calling thread.  Nothing is enqueued when a call fails
 *     its argument checks.
 */
#ifndef LIBPTYCHO_PTYCHO_H
#define LIBPTYCHO_PTYCHO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ptx_handle ptx_handle; /* opaque, owned by the library */

typedef enum {
    PTX_OK = 0,
    PTX_ERR_INVALID_ARG = 1,   /* null pointer, non-positive size, bad flag or name */
    PTX_ERR_UNSUPPORTED = 2,   /* frame size N not in the supported set, K > PTX_MAX_MODES */
    PTX_ERR_OUT_OF_BOUNDS = 3, /* a position puts its patch outside the object */
    PTX_ERR_CUDA = 4,          /* a CUDA runtime call failed (text in ptx_last_error) */
    PTX_ERR_TIMEOUT = 5,       /* a bounded device-side wait (tensor-copy arrival) of an earlier call
                                  gave up; that call's results are invalid; reported once */
    PTX_ERR_NOT_READY = 6      /* scratch too small or handle in an unusable state */
} ptx_status;

/* Flags of the cycle calls (bitwise OR). */
#define PTX_UPDATE_OBJ   0x1u  /* update the object (Psi2ObjProbe numerator N_O / denominator D_O) */
#define PTX_UPDATE_PROBE 0x2u  /* update the probe modes (N_P / D_P) */
#define PTX_DM_INIT_PSI  0x4u  /* DM only: set Psi = P . O[r_j] before the first cycle */
#define PTX_NO_NORMALISE 0x8u  /* accumulate N_O, D_O, N_P, D_P but do not normalise (data-parallel split) */
#define PTX_NO_GRAPH     0x10u /* enqueue kernels directly instead of replaying a captured CUDA graph */
#define PTX_UPDATE_BACKGROUND 0x40u /* AP only: update the incoherent background of the problems that have one */
/* Number format of the column pass's DFT stages (problems with N = 256 and one
 * mode: two 16-point stages; N = 512 with any number of modes: a 16-point and
 * a 32-point stage; other problems run FP32).  No PTX_FORM_* flag: the handle's
 * "tc" parameter (default FP32, the CUDA-core codelets).  At most one flag.
 * The tensor-core forms run each stage as tcgen05.mma GEMMs with the operands
 * split into terms of the narrow type and FP32 accumulation in TMEM:
 *   PTX_FORM_TF32X2  TF32 hi + lo, 3 products, about 2^-21 per product;
 *   PTX_FORM_BF16X3  BF16 hi + mid + lo, 6 products (every product down to
 *                    2^-16 of the result), the BF16 split that meets FP32 parity;
 *   PTX_FORM_BF16X2  BF16 hi + lo, 3 products, about 2^-16 per product: the
 *                    two-term split, below FP32 accuracy. */
#define PTX_FORM_TF32X2 0x1000u
#define PTX_FORM_BF16X3 0x2000u
#define PTX_FORM_BF16X2 0x4000u

#define PTX_MAX_MODES 8

/* Supported frame sizes N (N x N frames) the kernels are built for: products
 * of 2 and 3, and of 2 with 5 or 7 (the paper's FFT libraries accept prime
 * factors up to 7, Table 1 caption; 400^2 frames in Fig. 7). */
#define PTX_SUPPORTED_SIZES {8, 12, 16, 32, 64, 80, 128, 160, 192, 224, 256, 384, 400, 448, 512}

/* One ptychography problem (the paper's PtychoData plus the current Ptycho
 * object and probe, Section 4). */
typedef struct {
    int32_t N;              /* frame size: N x N detector pixels */
    int32_t K;              /* number of incoherent probe modes, 1..PTX_MAX_MODES */
    int32_t J;              /* number of scan positions (frames), >= 1 */
    int32_t Ho, Wo;         /* object height and width, each >= N */
    void* obj;              /* device complex64 [Ho][Wo]; updated in place by the cycles */
    void* probe;            /* device complex64 [K][N][N]; updated in place by the cycles */
    const int32_t* positions; /* host int32 [J][2] (row, col) top-left corners; copied at create;
                                 each must satisfy 0 <= row <= Ho-N, 0 <= col <= Wo-N */
    const float* iobs;      /* device float32 [J][N][N] observed intensities, FFT order; borrowed,
                               read-only, must stay valid for the handle's lifetime; negative
                               values are treated as 0.  iobs, probe and psi must be 16-byte
                               aligned and obj 8-byte aligned (PTX_ERR_INVALID_ARG otherwise) */
    const uint8_t* mask;    /* host uint8 [N][N], nonzero = bad pixel (left free by the projection,
                               excluded from the LLK and its gradient); NULL = no mask; copied */
    void* psi;              /* device complex64 [J][K][N][N] exit-wave stack Psi (the Ptycho
                               object's Psi array), needed by the AP and DM cycles; may be NULL
                               for LLK and ML */
    double nearfield;       /* 0: far field (the detector sees FT(Psi); iobs and mask in FFT
                               order).  c > 0: near field (PropagateNearField, paper Section 4
                               and the operator table): the detector sees IFT(FT(Psi) h),
                               h = exp(-i pi c (ky^2 + kx^2) / N^2) with signed frequencies,
                               c = lambda z / pixel^2; iobs and mask in detector pixels.  Near
                               field needs K = 1 and N >= 32 (PTX_ERR_UNSUPPORTED otherwise) and
                               serves the AP / DM cycles and ptx_llk, not the ML calls. */
    float* background;      /* device float32 [N][N] incoherent background B >= 0 (paper Section 4,
                               the Ptycho object's background), in the layout of iobs, or NULL.
                               When given, every frame's model intensity is I_c + B (LLK,
                               projection, gradient, line search) and AP cycles with
                               PTX_UPDATE_BACKGROUND replace B by B (1/J) sum_j I_o / (I_c + B)
                               on unmasked pixels (the update is multiplicative: start B > 0). */
} ptx_problem;

/* Device scratch needed by ptx_create for these problems, in bytes.  The caller
 * allocates it (e.g. with torch.empty) and keeps it alive until ptx_destroy.  It
 * holds the copied positions and mask, the Fourier-space work stack of one
 * batch of frames, the object / probe numerator-denominator accumulators and
 * the FP64 log-likelihood partial sums. */
ptx_status ptx_workspace_bytes(const ptx_problem* probs, int32_t nprob, size_t* scratch_bytes);

/* Create a handle for nprob problems (nprob = 1 for a single scan).  `probs` is
 * copied; the device arrays it points to are borrowed.  `scratch` is a device
 * buffer of at least ptx_workspace_bytes() bytes, 256-byte aligned.  Copies the
 * positions and the mask into scratch on `stream`, zeroes the accumulators and
 * waits for these copies (the only host synchronisation of the library).  Returns PTX_ERR_OUT_OF_BOUNDS for a position outside the
 * object, PTX_ERR_UNSUPPORTED for an unsupported N or K. */
ptx_status ptx_create(ptx_handle** out, const ptx_problem* probs, int32_t nprob,
                      void* scratch, size_t scratch_bytes, void* stream);

/* Alternating-projection cycles (the AP operator; Marchesini et al. 2013 as cited
 * in Section 4): per cycle, Phi = ObjProbe2Psi(O, P); Psi = IFT(ApplyAmplitude(FT(Phi)))
 * stored in probs[p].psi; then Psi2ObjProbe: the probe first,
 * P <- (N_P + d_P P) / (D_P + d_P), N_P = sum_j conj(O(r_j + x)) Psi_j(x),
 * D_P = sum_j |O(r_j + x)|^2, d_P = alpha_probe max D_P; then the object from the new
 * probe, O <- (N_O + d_O O) / (D_O + d_O), N_O = sum_j conj(P(x)) Psi_j(x) and
 * D_O = sum_j |P(x)|^2 at r = r_j + x, d_O = alpha_obj max D_O.  llk_dev: device double
 * [ncycles * nprob]; entry [c * nprob + p] receives the Poisson LLK (deviance form)
 * of FT(Phi) in cycle c of problem p.  Needs probs[p].psi. */
ptx_status ptx_ap_cycles(ptx_handle* h, int32_t ncycles, uint32_t flags, double* llk_dev, void* stream);

/* Difference-map cycles (the DM operator, beta = 1; Elser 2007 as cited in
 * Section 4): Phi = ObjProbe2Psi(O, P); X = 2 Phi - Psi;
 * Psi <- Psi + IFT(ApplyAmplitude(FT(X))) - Phi; then Psi2ObjProbe from the new Psi and
 * the normalisation as for AP.  Needs probs[p].psi.  With PTX_DM_INIT_PSI, Psi = Phi is
 * set at the first cycle.  llk_dev as for AP, with the LLK of FT(X). */
ptx_status ptx_dm_cycles(ptx_handle* h, int32_t ncycles, uint32_t flags, double* llk_dev, void* stream);

/* Algorithms of ptx_cycles. */
#define PTX_ALGO_AP 0
#define PTX_ALGO_DM 1

/* Cycles of a batched handle (nprob independent problems of any sizes), each
 * problem with its own algorithm: algorithms is a host int32 array [nprob] of
 * PTX_ALGO_AP / PTX_ALGO_DM.  One cycle is one CUDA graph over all problems: the
 * batches of every problem share the handle's lanes (streams), and a problem's
 * overlap update runs as soon as its own batches are done.  Semantics per
 * problem as ptx_ap_cycles / ptx_dm_cycles (PTX_DM_INIT_PSI applies to the DM
 * problems); llk_dev as there. */
ptx_status ptx_cycles(ptx_handle* h, int32_t ncycles, uint32_t flags, const int32_t* algorithms, double* llk_dev,
                      void* stream);

/* Exact Poisson log-likelihood of the current (O, P) (the LLK operator):
 * sum over frames and unmasked pixels of I_c - I_o + I_o ln(I_o / I_c) (I_c where
 * I_o = 0), I_c = sum_k |FT(Phi_jk)|^2.  Writes nprob doubles to llk_dev. */
ptx_status ptx_llk(ptx_handle* h, double* llk_dev, void* stream);

/* Gradient of the Poisson LLK with respect to the object and the probe (the
 * ML operator's gradient; Thibault & Guizar-Sicairos 2012 as cited in Section 4):
 * G = dL/dRe z + i dL/dIm z, i.e.
 *   G_O(r_j + x) = sum_jk conj(P_k(x)) IFT[w_j FT(Phi_jk)](x),
 *   G_Pk(x)      = sum_j conj(O(r_j + x)) IFT[w_j FT(Phi_jk)](x),
 *   w_j = 2 (1 - I_o / I_c) on unmasked pixels, 0 on masked ones.
 * grad_obj: device complex64 [Ho][Wo], grad_probe: device complex64 [K][N][N]
 * (problem 0; nprob must be 1), both overwritten.  Either may be NULL to skip it.
 * llk_dev (may be NULL) receives the LLK.  Psi is recomputed, never stored. */
ptx_status ptx_ml_grad(ptx_handle* h, void* grad_obj, void* grad_probe, double* llk_dev, void* stream);

/* Flag of ptx_ml_cycles: forget the previous gradient and direction first
 * (the next step is steepest descent). */
#define PTX_ML_RESTART 0x20u

/* Maximum-likelihood conjugate-gradient cycles on the Poisson LLK (the ML
 * operator; Thibault & Guizar-Sicairos 2012): per cycle the gradient G of
 * ptx_ml_grad (object and/or probe by PTX_UPDATE_OBJ / PTX_UPDATE_PROBE; the
 * paper's ML default updates the object only), the Polak-Ribiere direction
 * D <- -G + beta D with beta = max(0, (<G,G> - <G,Gp>) / <Gp,Gp>) (0 without a
 * previous gradient Gp; <a,b> = Re sum conj(a) b over object and probe), and the
 * step O += alpha D_O, P += alpha D_P with alpha = -L'(0) / L''(0) from the
 * expansion of the far field along the line (ptx_ml_line_coeffs), no step if
 * L''(0) <= 0.  The CG state lives in the handle's scratch and carries over
 * between calls.  llk_dev (may be NULL): device double [ncycles], the LLK before
 * each step.  nprob must be 1.  Runs entirely on the device (no host sync). */
ptx_status ptx_ml_cycles(ptx_handle* h, int32_t ncycles, uint32_t flags, double* llk_dev, void* stream);

/* Line-search coefficients of the ML step along (d_obj, d_probe) (device
 * complex64 [Ho][Wo] and [K][N][N]; either may be NULL = zero): with
 * FT((P + a dP)(O + a dO)) = A + a B + a^2 C, A = FT(P O), B = FT(dP O + P dO),
 * C = FT(dP dO), coeffs_dev[0] = L'(0) = sum (1 - I_o/I_c) dI and coeffs_dev[1] =
 * L''(0) = sum [(1 - I_o/I_c) d2I + (I_o/I_c^2) dI^2] over unmasked pixels, where
 * dI = 2 sum_k Re(conj(A) B) and d2I = 2 sum_k (|B|^2 + 2 Re(conj(A) C)).  FP64. */
ptx_status ptx_ml_line_coeffs(ptx_handle* h, const void* d_obj, const void* d_probe, double* coeffs_dev,
                              void* stream);

/* Stages of the second half of Psi2ObjProbe, for ptx_normalise. */
#define PTX_STAGE_PROBE         0x100u /* P <- (N_P + d_P P) / (D_P + d_P) from the probe accumulator, cleared */
#define PTX_STAGE_OBJ_GATHER    0x200u /* object accumulator <- N_O, D_O of this handle's frames, from the
                                          stored Psi' and the current probe */
#define PTX_STAGE_OBJ_NORMALISE 0x400u /* O <- (N_O + d_O O) / (D_O + d_O) from the object accumulator, cleared */

/* Run stages of the probe / object update after cycles run with PTX_NO_NORMALISE
 * (data-parallel split: all-reduce the probe accumulator, then PTX_STAGE_PROBE |
 * PTX_STAGE_OBJ_GATHER, all-reduce the object accumulator, then
 * PTX_STAGE_OBJ_NORMALISE).  PTX_UPDATE_PROBE selects PTX_STAGE_PROBE and
 * PTX_UPDATE_OBJ the two object stages. */
ptx_status ptx_normalise(ptx_handle* h, uint32_t flags, void* stream);

/* Device addresses of problem p's accumulators (for an all-reduce across GPUs):
 * obj_acc = float32 [Ho][Wo][4] {Re N_O, Im N_O, D_O, 0}; probe_acc = float32
 * [K][N][N][4] {Re N_Pk, Im N_Pk, D_P, 0}. */
ptx_status ptx_accumulators(ptx_handle* h, int32_t p, void** obj_acc, size_t* obj_acc_bytes,
                            void** probe_acc, size_t* probe_acc_bytes);

/* Set a scalar parameter: "alpha_obj" or "alpha_probe" (inertia factors of the
 * normalisation, default 0.01 each, must be >= 0); "lanes" (batches in flight per
 * cycle, 1..4, default 2); "batch_frames" (upper bound on frames per batch, 0 =
 * as many as the work stack holds); "bwd_slots" (frame slots of the row-backward
 * pass: blocks per row band, each looping over every bwd_slots-th frame of a
 * batch and flushing its probe sums once; 0, default: as many as are resident
 * at once); "persistent" (0, default; 1: the batch passes of every problem of
 * the handle run as the work items of one persistent launch per cycle, in
 * pipeline order over three work-stack slots, each item waiting (bounded)
 * for the items it depends on; for handles whose problems all have one probe
 * mode, N in {128, 192, 256, 384, 512}, far field and no background, others
 * keep the per-batch launches); "persistent_selftest" (1: the persistent
 * schedule's first column items wait for a forward item that never comes, so
 * their bounded wait gives up: the next cycle call returns PTX_ERR_TIMEOUT
 * once; for the tests of that failure path); "tc_selftest" (1: in the 256^2
 * tensor-core column pass one stage of the first frame issues no MMAs, so its
 * bounded wait (about 2^31 SM clocks) gives up and the next cycle call returns
 * PTX_ERR_TIMEOUT once; for the tests of that failure path); "tc_rows" (0,
 * default; 1: with a tensor-core form, the forward and backward row passes of
 * problems with N = 256 and one mode, or N = 512 and any number of modes, run
 * their DFT stages on the tensor cores too, so that every DFT stage of the
 * cycle is in that form); "pdl" (1, default: the FP32 register passes of
 * far-field problems without a background (forward row, column and backward
 * row passes of the one-mode AP / DM cycle within each lane, of ptx_llk,
 * ptx_ml_grad and the ML cycles' gradients; the one-mode line-search passes)
 * are launched as
 * programmatic dependents of the pass before them, so that a pass's first
 * blocks load their inputs while the previous pass's last blocks finish; 0:
 * plain launches, each pass after the whole previous one); "tma" (0, default:
 * the register column pass;
 * 1: the AP / DM column pass of one-mode problems with N = 256 takes its inputs
 * by 2D tensor copies (cp.async.bulk.tensor) in a persistent grid of two CTAs
 * per SM).  "tma_gather" (1, default: the object numerator / denominator of
 * frames with N >= 64 is gathered from boxes of Psi' and P brought into shared
 * memory by 3D tensor copies through a four-stage mbarrier ring; 0: the plain
 * gather).  "tc": the number format of the DFT stages of the AP / DM column
 * pass of problems with N = 256 and one mode or N = 512 (0, default: FP32 on the CUDA cores;
 * 1: TF32X2, 2: BF16X3, 3: BF16X2 on the tensor cores, as the PTX_FORM_*
 * cycle flags describe); a PTX_FORM_* flag of a cycle call overrides it for
 * that call.  Each pair of variants gives the same results up to rounding
 * (BF16X2: up to its larger rounding). */
ptx_status ptx_set_param(ptx_handle* h, const char* name, double value);

/* In-place orthonormal 2D FFT of `nframes` N x N complex64 frames (the FT
 * operator for direction = -1, IFT for direction = +1): X[ky][kx] =
 * (1/N) sum_{y,x} x[y][x] exp(direction * 2 pi i (ky y + kx x) / N).
 * data: device complex64 [nframes][N][N]. */
ptx_status ptx_fft2(void* data, int32_t nframes, int32_t N, int32_t direction, void* stream);

/* Kernel kinds reported by ptx_profile_read. */
#define PTX_KERNEL_ROW_FWD   0 /* gather x probe, (2 Phi - Psi), forward row FFT */
#define PTX_KERNEL_COL       1 /* column FFT, amplitude projection + LLK, inverse column FFT */
#define PTX_KERNEL_ROW_BWD   2 /* inverse row FFT, Psi update, probe numerator / denominator */
#define PTX_KERNEL_DEN_MAX   3 /* max of the denominators */
#define PTX_KERNEL_NORMALISE 4 /* normalisation of O and P */
#define PTX_KERNEL_CYCLE_END 5 /* FP64 LLK reduction of the cycle */
#define PTX_KERNEL_OBJ_GATHER 6 /* object numerator / denominator gathered per tile from Psi' */
#define PTX_KERNEL_KINDS     7

/* Position refinement (Psi2PosShift, paper Section 4, after Odstrcil et al.
 * 2018).  For every frame of problem p, the first-order least-squares shift
 * (row, col) in pixels that moves P . O[r_j] towards the projected exit wave
 * left in psi by the last AP cycle: with chi = Psi_j - P O[r_j] and
 * G_a = P dO/da (a = row, col; central differences of the object, one-sided on
 * its edges) it solves [<G_y,G_y> <G_y,G_x>; <G_x,G_y> <G_x,G_x>] d =
 * [<G_y,chi>; <G_x,chi>], <u,v> = sum over modes and pixels of Re(conj(u) v),
 * in FP64.  A frame whose gradient norm <G_y,G_y> + <G_x,G_x> is below
 * filter_ratio times the mean over frames (the paper's filter against weak
 * object gradients), or whose system is singular, gets (0, 0).
 * shifts: device float32 [J][2].  The positions themselves stay integer: the
 * caller accumulates the shifts and moves frames with ptx_set_positions. */
ptx_status ptx_position_shifts(ptx_handle* h, int32_t p, float filter_ratio, float* shifts, void* stream);

/* Replace the scan positions of problem p (host int32 [J][2], copied; the
 * same bounds as at create, PTX_ERR_OUT_OF_BOUNDS otherwise).  Rebuilds the
 * object tile lists in place and drops the captured cycle graphs; waits for
 * its copies (a host synchronisation). */
ptx_status ptx_set_positions(ptx_handle* h, int32_t p, const int32_t* positions, void* stream);

/* Per-kernel timing for measurement.  While enabled, the cycle calls launch
 * their kernels directly (no CUDA graph) and bracket every launch with CUDA
 * events recorded on the launch stream.  Enabling resets the counters. */
ptx_status ptx_profile_enable(ptx_handle* h, int32_t enable);

/* Wait for the recorded events and return, for each of the first `nkinds`
 * kernel kinds, the number of launches (host int64 array) and their summed
 * duration in milliseconds (host double array) since profiling was enabled. */
ptx_status ptx_profile_read(ptx_handle* h, int32_t nkinds, int64_t* launches, double* total_ms);

/* Size of the fixed device array used by ptx_llk_static. */
#define PTX_STATIC_SCRATCH_BYTES (16u << 20)

/* The exact Poisson log-likelihood of ptx_llk, computed without any device
 * allocation, for callers that cannot allocate: code embedded in a host
 * application that owns all device memory and hands out only its input and
 * output buffers, or a loop that must never enter an allocator (cudaMalloc,
 * torch's caching allocator).  The paper has no counterpart; this is a service
 * of this library.
 *
 * Inputs: obj device complex64 [Ho][Wo], probe device complex64 [K][N][N],
 * iobs device float32 [J][N][N] (FFT order), positions host int32 [J][2]
 * (row, col), mask host uint8 [N][N] or NULL; iobs and probe 16-byte aligned,
 * obj 8-byte aligned.  Output: llk_dev, one device
 * double.  No handle, no scratch argument: all working memory (copied
 * positions and mask, the Fourier work stack, the FP64 partial sums) lives in
 * one file-scope device array of PTX_STATIC_SCRATCH_BYTES (16 MiB) that every
 * GPU loading the library holds until the process exits.  Every call looks
 * up that array's address on the current device with cudaGetSymbolAddress
 * (no synchronisation).  The first call that sees an address on a device (the
 * first call there, or the first after a cudaDeviceReset reloaded the module)
 * also clears the array's mask region and synchronises the device once: make
 * that first call before any stream capture.  Sizes beyond the array (J > 65536, J * N / C > 65536 partial
 * sums with C columns per block of the column pass, or one frame's
 * K * N * N * 8-byte work stack larger than the array's
 * work region) are rejected with PTX_ERR_UNSUPPORTED and a message; nothing
 * is enqueued then.  All calls share the array and it keeps the last call's
 * contents; every call rewrites what it reads, but calls that overlap on the
 * GPU race on it.  Calls no cudaMalloc, cudaFree or allocating library routine. */
ptx_status ptx_llk_static(int32_t N, int32_t K, int32_t J, int32_t Ho, int32_t Wo, const void* obj,
                          const void* probe, const int32_t* positions, const float* iobs, const uint8_t* mask,
                          double* llk_dev, void* stream);

/* Photon counts to intensities: dst[i] = (float)src[i] for i < n, on the
 * device, asynchronous on the stream.  Detectors count photons as 16-bit
 * integers; uploading the counts and widening them on the device moves half
 * the bytes of a float32 upload (every uint16 value is exact in float32).
 * dst: device float32 [n] (e.g. a problem's iobs array, written in place),
 * src: device uint16 [n]; both 16-byte aligned.  n = 0 does nothing.
 * PTX_ERR_INVALID_ARG for a null or misaligned pointer. */
ptx_status ptx_counts_to_float(float* dst, const uint16_t* src, size_t n, void* stream);

/* Photon counts in one byte each plus an escape list: the compact exact form
 * of count frames whose counts are mostly below 255 (far-field frames are
 * mostly dark: at 1e6 photons per 256^2 frame 1.6 % of the pixels reach 255,
 * so the form moves 56 % of the bytes of uint16 counts).
 *
 * Host side (synchronous, no device work): out8[i] = min(src[i], 255) for
 * i < n, and for every i with src[i] >= 255, in increasing i, the escape
 * (esc_index[k], esc_value[k]) = (i, src[i]); *n_esc = the number of escapes.
 * src: host uint16 [n]; out8: host uint8 [n]; esc_index: host uint32 [cap];
 * esc_value: host uint16 [cap].  With cap = 0 and null out8, esc_index and
 * esc_value the call only counts the escapes.  PTX_ERR_OUT_OF_BOUNDS when the
 * escapes exceed cap (*n_esc still set, cap entries written);
 * PTX_ERR_INVALID_ARG for null arrays that are needed or n >= 2^32. */
ptx_status ptx_encode_counts8(const uint16_t* src, size_t n, uint8_t* out8, uint32_t* esc_index,
                              uint16_t* esc_value, size_t cap, size_t* n_esc);

/* Device side, asynchronous on the stream: dst[i] = (float)src8[i] for i < n,
 * then dst[esc_index[k]] = (float)esc_value[k] for k < n_esc (two kernels in
 * stream order), which restores the counts exactly.  dst: device float32 [n]
 * (e.g. a problem's iobs array), src8: device uint8 [n], both 16-byte
 * aligned; esc_index (uint32) and esc_value (uint16): device [n_esc], may be
 * null when n_esc = 0; an escape whose index is not below n is skipped.
 * n = 0 does nothing.
 * PTX_ERR_INVALID_ARG for a null or misaligned pointer or n >= 2^32. */
ptx_status ptx_counts8_to_float(float* dst, const uint8_t* src8, size_t n, const uint32_t* esc_index,
                                const uint16_t* esc_value, size_t n_esc, void* stream);

/* Self-test of the failure path of the bounded device waits (no GPU fault is
 * involved): enqueues one kernel whose single waiting thread waits for a flag
 * that nothing sets, for at most limit_us microseconds of the GPU's global
 * timer (1..1000000), and then records the give-up in the handle's device
 * error flag exactly as a cycle's tensor-copy wait that gives up does.  The
 * next ptx_ap_cycles / ptx_dm_cycles / ptx_cycles call on the handle, made
 * after the stream has passed the kernel, returns PTX_ERR_TIMEOUT once and
 * enqueues nothing; later calls work as before.  Returns PTX_OK when the
 * kernel is enqueued; PTX_ERR_INVALID_ARG for a null handle or a limit out of
 * range, PTX_ERR_NOT_READY when the handle has no error flag (mapped host
 * memory was unavailable at create). */
ptx_status ptx_wait_selftest(ptx_handle* h, int32_t limit_us, void* stream);

/* Number of kernel launches in one cycle of `algorithm` (PTX_ALGO_AP or
 * PTX_ALGO_DM, for every problem of the handle) with the cycle flags `flags`,
 * as the cycle's captured CUDA graph holds them (the graph is captured now if
 * it was not yet; call outside any stream capture).  A ptx_ap_cycles /
 * ptx_dm_cycles call adds one control kernel per call.  *count receives the
 * number (host).  PTX_ERR_INVALID_ARG for a null pointer or an unknown
 * algorithm. */
ptx_status ptx_cycle_kernels(ptx_handle* h, int32_t algorithm, uint32_t flags, int64_t* count);

/* FP32 fused multiply-add throughput probe (no counterpart in the paper; it
 * measures the ALU roof the FFT passes are compared against).  Enqueues
 * `blocks` blocks of 256 threads, each thread running `iters` rounds of 16
 * independent FMA chains, and writes one float per thread to `sink` (device
 * float32 [blocks * 256], caller-owned).  *flops (host) receives the floating-
 * point operations the launch performs (2 per FMA); time the launch with
 * events on `stream` and divide.  PTX_ERR_INVALID_ARG for blocks or iters < 1
 * or a null pointer. */
ptx_status ptx_fma_peak(int32_t blocks, int32_t iters, float* sink, double* flops, void* stream);

/* Position refinement, host step (paper Section 4: position refinement after
 * Odstrcil et al. 2018): the per-frame shifts of ptx_position_shifts (copied
 * to the host) accumulate into sub-pixel positions and frames move when their
 * rounded position changes.  For each frame j and axis a (row, col):
 *   pos_subpixel[j][a] = clip(pos_subpixel[j][a] + clip(step * shifts[j][a],
 *                             -max_shift, max_shift), 0, max_a)
 *   positions[j][a]    = nearest integer to pos_subpixel[j][a] (halves to even)
 * with max_row = Ho - N, max_col = Wo - N.  shifts: host float32 [J][2];
 * pos_subpixel: host float64 [J][2], in / out; positions: host int32 [J][2],
 * in (current) / out (new); *moved receives the number of frames whose integer
 * position changed (pass `positions` to ptx_set_positions when it is > 0).
 * Host only: touches no device memory and enqueues nothing.
 * PTX_ERR_INVALID_ARG for J < 0, a null pointer, or a negative bound. */
ptx_status ptx_accumulate_shifts(int32_t J, const float* shifts, double step, double max_shift, int32_t max_row,
                                 int32_t max_col, double* pos_subpixel, int32_t* positions, int32_t* moved);

/* Text of the last failure on the calling thread ("" if none). */
const char* ptx_last_error(void);

/* Destroy a handle (waits for nothing; the caller must make sure no call on it is
 * still running on the GPU before freeing the scratch).  NULL is ignored. */
void ptx_destroy(ptx_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* LIBPTYCHO_PTYCHO_H */
