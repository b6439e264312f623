// Register-resident DFT codelets and the shared-memory line FFT used by every
// pass of the ptychography cycle (the FT / IFT operators of the paper's operator
// table).  Transforms here are unnormalised: out[k] = sum_n in[n] w^(n k) with
// w = exp(DIR * 2 pi i / R), DIR = -1 forward, +1 inverse.  The orthonormal 1/N per
// 2D transform is applied by the callers in the elementwise steps.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace ptx {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cconjmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float cnorm(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
// a * (s i), s = +-1
template <int S>
__device__ __forceinline__ float2 mul_i(float2 a) {
    return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// Compile-time twiddles exp(2 pi i m / R).  cos/sin by Taylor series in double
// on the reduced angle; exact where the angle is a multiple of pi/4 so that the
// codelets skip trivial multiplications.
// ---------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846264338327950288;

__host__ __device__ constexpr double taylor_sin(double x) {
    double x2 = x * x, term = x, sum = x;
    for (int i = 1; i < 14; ++i) {
        term *= -x2 / double((2 * i) * (2 * i + 1));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int i = 1; i < 14; ++i) {
        term *= -x2 / double((2 * i - 1) * (2 * i));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr int pmod(int a, int b) { return ((a % b) + b) % b; }
// angle 2 pi m / R reduced to [-pi, pi)
__host__ __device__ constexpr double red_angle(int m, int R) {
    int mm = pmod(m, R);
    if (2 * mm >= R) mm -= R;
    return 2.0 * kPi * double(mm) / double(R);
}
__host__ __device__ constexpr double tw_cos(int m, int R) {
    return (pmod(4 * m, R) == 0) ? (pmod(m, R) == 0 ? 1.0 : (2 * pmod(m, R) == R ? -1.0 : 0.0))
                                 : taylor_cos(red_angle(m, R));
}
__host__ __device__ constexpr double tw_sin(int m, int R) {
    return (pmod(4 * m, R) == 0) ? ((4 * pmod(m, R) == R) ? 1.0 : ((4 * pmod(m, R) == 3 * R) ? -1.0 : 0.0))
                                 : taylor_sin(red_angle(m, R));
}

// v * exp(2 pi i m / R), specialised for the exact cases
template <int M, int R>
__device__ __forceinline__ float2 twiddle(float2 v) {
    constexpr int m = pmod(M, R);
    if constexpr (m == 0) {
        return v;
    } else if constexpr (4 * m == R) {
        return mul_i<1>(v);
    } else if constexpr (2 * m == R) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (4 * m == 3 * R) {
        return mul_i<-1>(v);
    } else if constexpr (pmod(8 * m, R) == 0) {
        // odd multiple of pi/4: (c + i s) with |c| = |s| = 1/sqrt(2)
        constexpr float h = 0.70710678118654752440f;
        constexpr float c = tw_cos(m, R) > 0 ? h : -h;
        constexpr float s = tw_sin(m, R) > 0 ? h : -h;
        // (x + i y)(c + i s) = (x c - y s) + i (x s + y c); with |c| = |s| = h
        float a = (c > 0) ? v.x : -v.x;
        float b = (s > 0) ? v.y : -v.y;
        float e = (s > 0) ? v.x : -v.x;
        float d = (c > 0) ? v.y : -v.y;
        return make_float2(h * (a - b), h * (e + d));
    } else {
        constexpr float c = (float)tw_cos(m, R);
        constexpr float s = (float)tw_sin(m, R);
        return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
    }
}

// ---------------------------------------------------------------------------
// Codelets: in-place unnormalised DFT of R registers, natural order in and out.
// ---------------------------------------------------------------------------
template <int R, int DIR>
struct Dft;

template <int DIR>
struct Dft<1, DIR> {
    __device__ __forceinline__ static void run(float2*) {}
};

template <int DIR>
struct Dft<2, DIR> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <int DIR>
struct Dft<3, DIR> {
    __device__ __forceinline__ static void run(float2* v) {
        // w = exp(DIR 2 pi i / 3) = -1/2 + DIR i sqrt(3)/2
        constexpr float h = 0.86602540378443864676f;
        float2 s = cadd(v[1], v[2]);
        float2 d = csub(v[1], v[2]);
        float2 m = make_float2(fmaf(-0.5f, s.x, v[0].x), fmaf(-0.5f, s.y, v[0].y));
        float2 r = mul_i<DIR>(cscale(d, h));
        v[0] = cadd(v[0], s);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
};

template <int DIR>
struct Dft<4, DIR> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 t0 = cadd(v[0], v[2]);
        float2 t1 = csub(v[0], v[2]);
        float2 t2 = cadd(v[1], v[3]);
        float2 t3 = mul_i<DIR>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

// Composite R = A * B: n = n1 + B n2, k = k2 + A k1.
//   X[k2 + A k1] = sum_n1 w_B^(n1 k1) [ w_R^(n1 k2) sum_n2 v[n1 + B n2] w_A^(n2 k2) ]
template <int A, int B, int DIR>
struct DftComposite {
    __device__ __forceinline__ static void run(float2* v) {
        constexpr int R = A * B;
        float2 y[R];  // y[n1 * A + k2]
#pragma unroll
        for (int n1 = 0; n1 < B; ++n1) {
            float2 t[A];
#pragma unroll
            for (int n2 = 0; n2 < A; ++n2) t[n2] = v[n1 + B * n2];
            Dft<A, DIR>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < A; ++k2) y[n1 * A + k2] = t[k2];
        }
        apply_tw(y, std::integral_constant<int, 0>());
#pragma unroll
        for (int k2 = 0; k2 < A; ++k2) {
            float2 t[B];
#pragma unroll
            for (int n1 = 0; n1 < B; ++n1) t[n1] = y[n1 * A + k2];
            Dft<B, DIR>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < B; ++k1) v[k2 + A * k1] = t[k1];
        }
    }
    // y[n1*A + k2] *= w_R^(DIR n1 k2), unrolled at compile time
    template <int I>
    __device__ __forceinline__ static void apply_tw(float2* y, std::integral_constant<int, I>) {
        if constexpr (I < A * B) {
            constexpr int n1 = I / A, k2 = I % A;
            y[I] = twiddle<DIR * n1 * k2, A * B>(y[I]);
            apply_tw(y, std::integral_constant<int, I + 1>());
        }
    }
};

// Prime R (5, 7): the DFT written out, out[k] = v[0] + sum_{n>0} v[n] w^(n k),
// pairing n and R - n so that each pair costs one complex sum and one
// difference: out[k] = v0 + sum_{n<=R/2} [(v_n + v_{R-n}) cos(2 pi n k / R)
// + i DIR (v_n - v_{R-n}) sin(2 pi n k / R)].
template <int R, int DIR>
struct DftPrime {
    __device__ __forceinline__ static void run(float2* v) {
        constexpr int H = R / 2;
        float2 sp[H], sm[H];
#pragma unroll
        for (int n = 1; n <= H; ++n) {
            sp[n - 1] = cadd(v[n], v[R - n]);
            sm[n - 1] = csub(v[n], v[R - n]);
        }
        float2 out[R];
        float2 dc = v[0];
#pragma unroll
        for (int n = 0; n < H; ++n) dc = cadd(dc, sp[n]);
        out[0] = dc;
        apply<1>(v[0], sp, sm, out);
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = out[k];
    }
    template <int K>
    __device__ __forceinline__ static void apply(float2 v0, const float2* sp, const float2* sm, float2* out) {
        if constexpr (K <= R / 2) {
            constexpr int H = R / 2;
            float2 re = v0, im = make_float2(0.f, 0.f);
            term<K, 1>(sp, sm, re, im);
            // out[K] = re + i DIR im, out[R - K] = re - i DIR im
            const float2 t = mul_i<DIR>(im);
            out[K] = cadd(re, t);
            out[R - K] = csub(re, t);
            (void)H;
            apply<K + 1>(v0, sp, sm, out);
        }
    }
    template <int K, int N1>
    __device__ __forceinline__ static void term(const float2* sp, const float2* sm, float2& re, float2& im) {
        if constexpr (N1 <= R / 2) {
            constexpr float c = (float)tw_cos(N1 * K, R);
            constexpr float s = (float)tw_sin(N1 * K, R);
            re = make_float2(fmaf(sp[N1 - 1].x, c, re.x), fmaf(sp[N1 - 1].y, c, re.y));
            im = make_float2(fmaf(sm[N1 - 1].x, s, im.x), fmaf(sm[N1 - 1].y, s, im.y));
            term<K, N1 + 1>(sp, sm, re, im);
        }
    }
};
template <int DIR> struct Dft<5, DIR> : DftPrime<5, DIR> {};
template <int DIR> struct Dft<7, DIR> : DftPrime<7, DIR> {};
template <int DIR> struct Dft<6, DIR> : DftComposite<3, 2, DIR> {};
template <int DIR> struct Dft<10, DIR> : DftComposite<5, 2, DIR> {};
template <int DIR> struct Dft<14, DIR> : DftComposite<7, 2, DIR> {};
template <int DIR> struct Dft<20, DIR> : DftComposite<5, 4, DIR> {};
template <int DIR> struct Dft<28, DIR> : DftComposite<7, 4, DIR> {};
template <int DIR> struct Dft<25, DIR> : DftComposite<5, 5, DIR> {};
template <int DIR> struct Dft<8, DIR> : DftComposite<4, 2, DIR> {};
template <int DIR> struct Dft<12, DIR> : DftComposite<4, 3, DIR> {};
template <int DIR> struct Dft<16, DIR> : DftComposite<4, 4, DIR> {};
template <int DIR> struct Dft<24, DIR> : DftComposite<8, 3, DIR> {};
template <int DIR> struct Dft<32, DIR> : DftComposite<8, 4, DIR> {};

// ---------------------------------------------------------------------------
// Line-FFT plan: N = R * M.  Pass 1 runs M-way parallel R-point codelets on
// x[n1 + M n2], twiddles by w_N^(n1 k2) and writes y[k2 (M+1) + n1] (padded);
// pass 2 runs R-way parallel M-point codelets and writes X[k2 + R k1] (natural).
// ---------------------------------------------------------------------------
template <int N> struct Plan;
template <> struct Plan<8>   { static constexpr int R = 8,  M = 1;  };
template <> struct Plan<12>  { static constexpr int R = 12, M = 1;  };
template <> struct Plan<16>  { static constexpr int R = 16, M = 1;  };
template <> struct Plan<32>  { static constexpr int R = 8,  M = 4;  };
template <> struct Plan<64>  { static constexpr int R = 8,  M = 8;  };
template <> struct Plan<128> { static constexpr int R = 16, M = 8;  };
template <> struct Plan<192> { static constexpr int R = 16, M = 12; };
template <> struct Plan<256> { static constexpr int R = 16, M = 16; };
template <> struct Plan<384> { static constexpr int R = 16, M = 24; };
template <> struct Plan<512> { static constexpr int R = 16, M = 32; };
// sizes with factors 5 and 7 (the paper's FFT libraries accept radix up to 7)
template <> struct Plan<80>  { static constexpr int R = 10, M = 8;  };
template <> struct Plan<160> { static constexpr int R = 16, M = 10; };
template <> struct Plan<224> { static constexpr int R = 16, M = 14; };
template <> struct Plan<400> { static constexpr int R = 16, M = 25; };
template <> struct Plan<448> { static constexpr int R = 16, M = 28; };

// Line pitch (in complex elements) in shared memory: room for the padded
// intermediate layout, and odd so that column-major accesses are conflict-free.
template <int N>
__host__ __device__ constexpr int line_pitch() {
    return Plan<N>::M == 1 ? N + 1 : N + Plan<N>::R + 1;
}

// Twiddle table layout (forward sign): tw[k2 * M + n1] = exp(-2 pi i n1 k2 / N).
// In-place FFT of `nlines` lines (each N contiguous elements, pitch line_pitch<N>())
// held in shared memory by a block of T threads.  MAXLINES bounds nlines at
// compile time (register arrays).  Ends with a __syncthreads().
template <int N, int DIR, int T, int MAXLINES>
__device__ __forceinline__ void fft_lines(float2* __restrict__ buf, int nlines, const float2* __restrict__ tw) {
    constexpr int R = Plan<N>::R;
    constexpr int M = Plan<N>::M;
    constexpr int P = line_pitch<N>();
    const int tid = threadIdx.x;
    if constexpr (M == 1) {
        constexpr int I = (MAXLINES + T - 1) / T;
#pragma unroll
        for (int i = 0; i < I; ++i) {
            int line = tid + i * T;
            if (line < nlines) {
                float2 v[N];
                float2* p = buf + line * P;
#pragma unroll
                for (int n = 0; n < N; ++n) v[n] = p[n];
                Dft<N, DIR>::run(v);
#pragma unroll
                for (int n = 0; n < N; ++n) p[n] = v[n];
            }
        }
        __syncthreads();
    } else {
        constexpr int I1 = (MAXLINES * M + T - 1) / T;
        constexpr int I2 = (MAXLINES * R + T - 1) / T;
        // pass 1: load
        float2 v[I1][R];
#pragma unroll
        for (int i = 0; i < I1; ++i) {
            int w = tid + i * T;
            if (w < nlines * M) {
                int line = w / M, n1 = w - line * M;
                const float2* p = buf + line * P + n1;
#pragma unroll
                for (int n2 = 0; n2 < R; ++n2) v[i][n2] = p[M * n2];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < I1; ++i) {
            int w = tid + i * T;
            if (w < nlines * M) {
                int line = w / M, n1 = w - line * M;
                Dft<R, DIR>::run(v[i]);
                float2* p = buf + line * P + n1;
                p[0] = v[i][0];
#pragma unroll
                for (int k2 = 1; k2 < R; ++k2) {
                    float2 t = tw[k2 * M + n1];
                    if (DIR > 0) t.y = -t.y;
                    p[k2 * (M + 1)] = cmul(v[i][k2], t);
                }
            }
        }
        __syncthreads();
        // pass 2
        float2 u[I2][M];
#pragma unroll
        for (int i = 0; i < I2; ++i) {
            int w = tid + i * T;
            if (w < nlines * R) {
                int line = w / R, k2 = w - line * R;
                const float2* p = buf + line * P + k2 * (M + 1);
#pragma unroll
                for (int n1 = 0; n1 < M; ++n1) u[i][n1] = p[n1];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < I2; ++i) {
            int w = tid + i * T;
            if (w < nlines * R) {
                int line = w / R, k2 = w - line * R;
                Dft<M, DIR>::run(u[i]);
                float2* p = buf + line * P + k2;
#pragma unroll
                for (int k1 = 0; k1 < M; ++k1) p[R * k1] = u[i][k1];
            }
        }
        __syncthreads();
    }
}

}  // namespace ptx
