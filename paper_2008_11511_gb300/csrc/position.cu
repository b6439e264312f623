// Position refinement (Psi2PosShift): per frame the first-order least-squares
// shift between the model exit wave Phi_j = P O[r_j] and the projected wave
// Psi_j left by the last AP / DM cycle.  With chi = Psi_j - Phi_j and
// G_a = P dO/da (a = y, x; central differences of the object, one-sided on its
// edges), the 2 x 2 normal equations
//   [<G_y,G_y> <G_y,G_x>; <G_x,G_y> <G_x,G_x>] d = [<G_y,chi>; <G_x,chi>],
// <u,v> = sum over modes and pixels of Re(conj(u) v), give d = (d_y, d_x).
// A frame whose gradient norm <G_y,G_y> + <G_x,G_x> is below filter_ratio
// times the mean over frames (or whose system is singular) keeps its position.
#include "kernels.cuh"

namespace ptx {

namespace {

__device__ __forceinline__ float2 obj_at(const ProbArgs& a, int y, int x) { return a.obj[(size_t)y * a.Wo + x]; }

// dO/dy, dO/dx at (y, x) of the object
__device__ __forceinline__ void obj_grad(const ProbArgs& a, int y, int x, float2& gy, float2& gx) {
    const int y0 = y > 0 ? y - 1 : y, y1 = y < a.Ho - 1 ? y + 1 : y;
    const int x0 = x > 0 ? x - 1 : x, x1 = x < a.Wo - 1 ? x + 1 : x;
    const float sy = 1.0f / (float)(y1 - y0), sx = 1.0f / (float)(x1 - x0);
    gy = cscale(csub(obj_at(a, y1, x), obj_at(a, y0, x)), sy);
    gx = cscale(csub(obj_at(a, y, x1), obj_at(a, y, x0)), sx);
}

}  // namespace

// grid (rows / 8 bands, J): block sums the five products of its 8 rows of frame j
// over all modes and writes them to part[(j * bands + band) * 5 + q] (FP64).
__global__ void __launch_bounds__(256) k_pos_sums(ProbArgs a, double* part) {
    __shared__ double red[5][8];
    const int N = a.N, K = a.K;
    const int band = blockIdx.x, j = blockIdx.y;
    const int2 p = a.pos[j];
    float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // yy, yx, xx, y.chi, x.chi
    for (int e = threadIdx.x; e < 8 * N; e += blockDim.x) {
        const int y = band * 8 + e / N, x = e % N;
        if (y >= N) break;
        float2 gy, gx;
        obj_grad(a, p.x + y, p.y + x, gy, gx);
        const float2 o = obj_at(a, p.x + y, p.y + x);
        for (int k = 0; k < K; ++k) {
            const size_t pix = ((size_t)k * N + y) * N + x;
            const float2 pr = __ldg(a.probe + pix);
            const float2 chi = csub(a.psi[(size_t)j * K * N * N + pix], cmul(pr, o));
            const float2 Gy = cmul(pr, gy), Gx = cmul(pr, gx);
            s[0] += cnorm(Gy);
            s[1] += Gy.x * Gx.x + Gy.y * Gx.y;
            s[2] += cnorm(Gx);
            s[3] += Gy.x * chi.x + Gy.y * chi.y;
            s[4] += Gx.x * chi.x + Gx.y * chi.y;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double v = (double)s[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        part[((size_t)j * gridDim.x + band) * 5 + threadIdx.x] = v;
    }
}

// One block: per-frame sums in band order, the mean gradient norm, the solves.
__global__ void __launch_bounds__(1024) k_pos_solve(const double* part, int J, int bands, float filter_ratio,
                                                    float* shifts) {
    __shared__ double red[32];
    double nsum = 0.0;
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        double yy = 0.0, xx = 0.0;
        for (int b = 0; b < bands; ++b) {
            yy += part[((size_t)j * bands + b) * 5 + 0];
            xx += part[((size_t)j * bands + b) * 5 + 2];
        }
        nsum += yy + xx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nsum += __shfl_down_sync(0xffffffffu, nsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nsum;
    __syncthreads();
    double total = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) total += red[w];
    const double mean = total / (double)J;
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        double m[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int b = 0; b < bands; ++b)
            for (int q = 0; q < 5; ++q) m[q] += part[((size_t)j * bands + b) * 5 + q];
        const double norm = m[0] + m[2];
        const double det = m[0] * m[2] - m[1] * m[1];
        float dy = 0.f, dx = 0.f;
        if (norm >= (double)filter_ratio * mean && det > 1e-12 * norm * norm) {
            dy = (float)((m[2] * m[3] - m[1] * m[4]) / det);
            dx = (float)((m[0] * m[4] - m[1] * m[3]) / det);
        }
        shifts[2 * j] = dy;
        shifts[2 * j + 1] = dx;
    }
}

}  // namespace ptx
