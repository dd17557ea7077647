// Batched power-of-two FFT building blocks for sm_103a (CUDA cores, FP32).
//
// Every transform of length L is held by T = L / P threads, P points per thread, in the
// "cyclic" layout: thread i holds x[i + T*u], u = 0..P-1.  A transform is computed in two
// register passes (four-step factorisation L = P * T, T <= P):
//   pass 1: P-point DFT over u inside each thread, twiddle w_L^{i*k1};
//   one exchange through shared memory;
//   pass 2: T-point DFTs over the threads, P/T of them per thread;
// and the result comes back in the same cyclic layout: thread i holds X[i + T*u].
//
// Shared memory of QT transforms is interleaved ([index][transform]) so that the lanes of
// a warp, which run consecutive transforms, touch consecutive words (conflict-free).
//
// Twiddles inside a thread are compile-time constants evaluated by constexpr code below
// (Taylor series after exact argument reduction); the pass twiddles come from a table
// built on the host in double precision.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace ddm {

// ------------------------------------------------------------------ constexpr trig
// cos and sin of 2*pi*a/b for integers, reduced exactly to an angle in [0, pi/4] and
// evaluated by Taylor series in double precision (|error| < 1e-17 there).
__host__ __device__ constexpr double cx_taylor_sin(double x) {
    double term = x, sum = x;
    for (int n = 1; n < 14; ++n) {
        term *= -x * x / (double)((2 * n) * (2 * n + 1));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double cx_taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int n = 1; n < 14; ++n) {
        term *= -x * x / (double)((2 * n - 1) * (2 * n));
        sum += term;
    }
    return sum;
}
constexpr double kPi = 3.14159265358979323846264338327950288;

// returns {cos, sin} of 2*pi*a/b
struct cx_cs { double c, s; };
__host__ __device__ constexpr cx_cs cx_cossin_frac(long a, long b) {
    // reduce a/b to [0, 1)
    long r = a % b;
    if (r < 0) r += b;
    // octant: angle = 2*pi*r/b, work with eighths: 8r/b
    const long e8 = 8 * r;                 // angle in units of pi/4 is e8 / b
    const long oct = e8 / b;               // 0..7
    const long rem = e8 - oct * b;         // remainder in [0, b)
    // angle within the octant in radians: (rem / b) * pi/4
    const double x = (double)rem / (double)b * (kPi / 4.0);
    const double sx = cx_taylor_sin(x), cxv = cx_taylor_cos(x);
    const double sy = cx_taylor_sin(kPi / 4.0 - x), cy = cx_taylor_cos(kPi / 4.0 - x);
    // angle = oct * pi/4 + x
    switch (oct) {
        case 0: return {cxv, sx};
        case 1: return {sy, cy};            // pi/2 - (pi/4 - x)
        case 2: return {-sx, cxv};          // pi/2 + x
        case 3: return {-cy, sy};           // pi - (pi/4 - x)
        case 4: return {-cxv, -sx};         // pi + x
        case 5: return {-sy, -cy};          // 3pi/2 - (pi/4 - x)
        case 6: return {sx, -cxv};          // 3pi/2 + x
        default: return {cy, -sy};          // 2pi - (pi/4 - x)
    }
}

// Returns p unchanged but hides its value from the optimiser, so that addresses derived
// from it are recomputed where they are used instead of being kept live in registers
// across a transform (32 strided addresses would otherwise pin 64 registers).
template <typename T>
__device__ __forceinline__ T* opaque_ptr(T* p) {
    asm volatile("" : "+l"(p));
    return p;
}

// Compiler-only memory fence: shared/global loads may not be hoisted across it.  Used
// every few elements in unrolled element-wise loops so the scheduler does not pull all
// of a thread's table loads up front and run out of registers.
__device__ __forceinline__ void hoist_fence() { asm volatile("" ::: "memory"); }

// ------------------------------------------------------------------ paired FP32
// Blackwell executes two FP32 additions or FMAs in one instruction (PTX add/sub/fma
// .rn.f32x2 on a 64-bit register pair).  Each lane rounds exactly as the scalar
// instruction does, so results are bitwise those of the scalar code; only the number of
// issued instructions changes.  DDM_PAIRED selects how much of the complex arithmetic uses
// them: 0 none, 1 complex additions, 2 also the two FMAs that finish a general butterfly.
#ifndef DDM_PAIRED
#define DDM_PAIRED 2
#endif
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 r;
    asm("{\n .reg .b64 ra, rb, rr;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " add.rn.f32x2 rr, ra, rb;\n mov.b64 {%0, %1}, rr;\n}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 r;
    asm("{\n .reg .b64 ra, rb, rr;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " sub.rn.f32x2 rr, ra, rb;\n mov.b64 {%0, %1}, rr;\n}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
// a * b + c, lane by lane
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{\n .reg .b64 ra, rb, rc, rr;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " mov.b64 rc, {%6, %7};\n fma.rn.f32x2 rr, ra, rb, rc;\n mov.b64 {%0, %1}, rr;\n}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}

// ------------------------------------------------------------------ complex helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#if DDM_PAIRED >= 1
    return add2(a, b);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
#if DDM_PAIRED >= 1
    return sub2(a, b);
#else
    return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
__device__ __forceinline__ float2 cmul_conj(float2 a, float2 w) {   // a * conj(w)
    return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// multiply by w_R^K (forward: exp(-2 pi i K / R); inverse: the conjugate), K constant
template <int R, int K, bool INV>
__device__ __forceinline__ float2 twiddle_const(float2 o) {
    constexpr int k = ((K % R) + R) % R;
    if constexpr (k == 0) {
        return o;
    } else if constexpr (4 * k == R) {                 // -i (forward), +i (inverse)
        return INV ? make_float2(-o.y, o.x) : make_float2(o.y, -o.x);
    } else if constexpr (2 * k == R) {
        return make_float2(-o.x, -o.y);
    } else if constexpr (4 * k == 3 * R) {             // +i (forward), -i (inverse)
        return INV ? make_float2(o.y, -o.x) : make_float2(-o.y, o.x);
    } else if constexpr (8 * k == R) {                 // (1 -/+ i)/sqrt2
        constexpr float h = (float)cx_cossin_frac(1, 8).c;
        return INV ? make_float2((o.x - o.y) * h, (o.x + o.y) * h)
                   : make_float2((o.x + o.y) * h, (o.y - o.x) * h);
    } else if constexpr (8 * k == 3 * R) {             // (-1 -/+ i)/sqrt2
        constexpr float h = (float)cx_cossin_frac(1, 8).c;
        return INV ? make_float2(-(o.x + o.y) * h, (o.x - o.y) * h)
                   : make_float2((o.y - o.x) * h, -(o.x + o.y) * h);
    } else {
        constexpr cx_cs cs = cx_cossin_frac(k, R);
        constexpr float c = (float)cs.c;
        constexpr float s = INV ? (float)cs.s : (float)-cs.s;
        return make_float2(fmaf(o.x, c, -o.y * s), fmaf(o.x, s, o.y * c));
    }
}

// e + w o and e - w o for the constant twiddle w = w_R^K.  A general twiddle is applied in
// factored form, w o = c (o.x - t o.y, o.y + t o.x) with t = s / c (or the same with s
// factored out when |s| > |c|, so that |t| <= 1): two FMAs build the bracket and four
// more finish both outputs, six FMA-pipe instructions instead of eight.
__host__ __device__ constexpr double cx_absd(double x) { return x < 0 ? -x : x; }

template <int R, int K, bool INV>
__device__ __forceinline__ void bfly_const(float2 e, float2 o, float2& lo, float2& hi) {
    constexpr int k = ((K % R) + R) % R;
    if constexpr (k == 0 || 4 * k == R || 2 * k == R || 4 * k == 3 * R) {
        const float2 t = twiddle_const<R, K, INV>(o);
        lo = cadd(e, t);
        hi = csub(e, t);
    } else {
        constexpr cx_cs cs = cx_cossin_frac(k, R);
        constexpr double c = cs.c;
        constexpr double s = INV ? cs.s : -cs.s;
        if constexpr (cx_absd(c) >= cx_absd(s)) {
            constexpr float cf = (float)c;
            constexpr float tf = (float)(s / c);
            const float ux = fmaf(-tf, o.y, o.x), uy = fmaf(tf, o.x, o.y);
#if DDM_PAIRED >= 2
            const float2 u = make_float2(ux, uy);
            lo = fma2(u, make_float2(cf, cf), e);
            hi = fma2(u, make_float2(-cf, -cf), e);
#else
            lo = make_float2(fmaf(cf, ux, e.x), fmaf(cf, uy, e.y));
            hi = make_float2(fmaf(-cf, ux, e.x), fmaf(-cf, uy, e.y));
#endif
        } else {
            constexpr float sf = (float)s;
            constexpr float tf = (float)(c / s);
            const float ux = fmaf(tf, o.x, -o.y), uy = fmaf(tf, o.y, o.x);
#if DDM_PAIRED >= 2
            const float2 u = make_float2(ux, uy);
            lo = fma2(u, make_float2(sf, sf), e);
            hi = fma2(u, make_float2(-sf, -sf), e);
#else
            lo = make_float2(fmaf(sf, ux, e.x), fmaf(sf, uy, e.y));
            hi = make_float2(fmaf(-sf, ux, e.x), fmaf(-sf, uy, e.y));
#endif
        }
    }
}

// ------------------------------------------------------------------ in-register DFT
// Unnormalised DFT of R = 2^n points held in registers, natural order in and out.
// Radix-2 decimation in time with compile-time twiddles; radix-4 leaves.
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2* v);

template <int R, bool INV, int... K>
__device__ __forceinline__ void dit_combine(float2* v, const float2* e, const float2* o,
                                            std::integer_sequence<int, K...>) {
    (bfly_const<R, K, INV>(e[K], o[K], v[K], v[K + R / 2]), ...);
}

template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2* v) {
    if constexpr (R == 1) {
        return;
    } else if constexpr (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        const float2 s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
        const float2 r = twiddle_const<4, 1, INV>(d13);
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, r);
        v[3] = csub(d02, r);
    } else {
        float2 e[R / 2], o[R / 2];
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            e[k] = v[2 * k];
            o[k] = v[2 * k + 1];
        }
        dft_reg<R / 2, INV>(e);
        dft_reg<R / 2, INV>(o);
        dit_combine<R, INV>(v, e, o, std::make_integer_sequence<int, R / 2>{});
    }
}

// ------------------------------------------------------------------ mixed radix (2, 3, 5)
// DFTs of 3 and 5 points in place.  s i z below is -i z (forward) or +i z (inverse).
template <bool INV>
__device__ __forceinline__ float2 times_si(float2 z) {
    return INV ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
}
template <bool INV>
__device__ __forceinline__ void dft3(float2& a, float2& b, float2& c) {
    constexpr float h = (float)cx_cossin_frac(1, 3).s;           // sin(2 pi / 3)
    const float2 t1 = cadd(b, c), d = csub(b, c);
    const float2 t2 = make_float2(fmaf(-0.5f, t1.x, a.x), fmaf(-0.5f, t1.y, a.y));
    const float2 m = times_si<INV>(make_float2(h * d.x, h * d.y));
    a = cadd(a, t1);
    b = cadd(t2, m);
    c = csub(t2, m);
}
template <bool INV>
__device__ __forceinline__ void dft5(float2& a, float2& b, float2& c, float2& d, float2& e) {
    constexpr float c1 = (float)cx_cossin_frac(1, 5).c, c2 = (float)cx_cossin_frac(2, 5).c;
    constexpr float s1 = (float)cx_cossin_frac(1, 5).s, s2 = (float)cx_cossin_frac(2, 5).s;
    const float2 t1 = cadd(b, e), t2 = cadd(c, d), t3 = csub(b, e), t4 = csub(c, d);
    const float2 r1 = make_float2(fmaf(c2, t2.x, fmaf(c1, t1.x, a.x)), fmaf(c2, t2.y, fmaf(c1, t1.y, a.y)));
    const float2 r2 = make_float2(fmaf(c1, t2.x, fmaf(c2, t1.x, a.x)), fmaf(c1, t2.y, fmaf(c2, t1.y, a.y)));
    const float2 m1 = times_si<INV>(make_float2(fmaf(s2, t4.x, s1 * t3.x), fmaf(s2, t4.y, s1 * t3.y)));
    const float2 m2 = times_si<INV>(make_float2(fmaf(-s1, t4.x, s2 * t3.x), fmaf(-s1, t4.y, s2 * t3.y)));
    a = cadd(a, cadd(t1, t2));
    b = cadd(r1, m1);
    e = csub(r1, m1);
    c = cadd(r2, m2);
    d = csub(r2, m2);
}

// Unnormalised DFT of N = 2^a 3^b 5^c points in registers, natural order in and out:
// decimation in time by the prime p (5, then 3, then the power-of-two dft_reg), the p
// sub-sequences v[p j + r] transformed, then for every k < N/p the twiddles w_N^{r k}
// (compile-time constants) and a p-point DFT give X[k + (N/p) q], q < p.
template <int N, bool INV>
__device__ __forceinline__ void dft_mix(float2* v);

template <int N, int P, int K, bool INV>
__device__ __forceinline__ void mix_combine_k(float2* v, float2 (*sub)[N / P]) {
    constexpr int M = N / P;
    if constexpr (P == 5) {
        float2 a = sub[0][K], b = twiddle_const<N, K, INV>(sub[1][K]), c = twiddle_const<N, 2 * K, INV>(sub[2][K]);
        float2 d = twiddle_const<N, 3 * K, INV>(sub[3][K]), e = twiddle_const<N, 4 * K, INV>(sub[4][K]);
        dft5<INV>(a, b, c, d, e);
        v[K] = a; v[K + M] = b; v[K + 2 * M] = c; v[K + 3 * M] = d; v[K + 4 * M] = e;
    } else if constexpr (P == 3) {
        float2 a = sub[0][K], b = twiddle_const<N, K, INV>(sub[1][K]), c = twiddle_const<N, 2 * K, INV>(sub[2][K]);
        dft3<INV>(a, b, c);
        v[K] = a; v[K + M] = b; v[K + 2 * M] = c;
    }
}
template <int N, int P, bool INV, int... K>
__device__ __forceinline__ void mix_combine(float2* v, float2 (*sub)[N / P], std::integer_sequence<int, K...>) {
    (mix_combine_k<N, P, K, INV>(v, sub), ...);
}

template <int N, bool INV>
__device__ __forceinline__ void dft_mix(float2* v) {
    if constexpr ((N & (N - 1)) == 0) {
        dft_reg<N, INV>(v);
    } else {
        constexpr int P = (N % 5 == 0) ? 5 : 3;
        static_assert(N % P == 0, "dft_mix: lengths 2^a 3^b 5^c");
        constexpr int M = N / P;
        float2 sub[P][M];
#pragma unroll
        for (int r = 0; r < P; ++r)
#pragma unroll
            for (int j = 0; j < M; ++j) sub[r][j] = v[P * j + r];
#pragma unroll
        for (int r = 0; r < P; ++r) dft_mix<M, INV>(sub[r]);
        mix_combine<N, P, INV>(v, sub, std::make_integer_sequence<int, M>{});
    }
}

// ------------------------------------------------------------------ two-pass FFT
template <int L>
struct FftShape {
    static_assert((L & (L - 1)) == 0 && L >= 1 && L <= 1024, "L must be a power of two <= 1024");
    static constexpr int P = L < 32 ? L : 32;   // points per thread
    static constexpr int T = L / P;              // threads per transform
    static_assert(T <= P, "two-pass factorisation needs T <= P");
};

// Host/device twiddle table for the pass between the two register passes of an L-point
// transform: tw[k1 * T + i] = exp(-2 pi i * i * k1 / L), k1 < P, i < T (L entries).
inline void host_pass_twiddles(int L, float2* out) {
    const int P = L < 32 ? L : 32, T = L / P;
    for (int k1 = 0; k1 < P; ++k1)
        for (int i = 0; i < T; ++i) {
            const cx_cs cs = cx_cossin_frac((long)((long)i * k1 % L), L);
            out[k1 * T + i] = make_float2((float)cs.c, (float)-cs.s);
        }
}

// Shared-memory placement of the logical exchange index idx (0..L-1) of one transform.
// Interleaved: QT transforms side by side, lanes of a warp on consecutive transforms.
template <int QT>
struct AddrInterleaved {
    int ql;
    __device__ __forceinline__ int operator()(int idx) const { return idx * QT + ql; }
    template <int T>
    __device__ __forceinline__ int at(int hi, int lo) const { return (hi * T + lo) * QT + ql; }
};
// Transform-major with one pad element per T: lanes of a warp on consecutive i.
template <int L>
struct AddrPadded {
    int base;   // transform index * stride()
    static constexpr int T = FftShape<L>::T;
    static constexpr int stride() { return L + L / T; }
    __device__ __forceinline__ int operator()(int idx) const { return base + idx + idx / T; }
    template <int T_>
    __device__ __forceinline__ int at(int hi, int lo) const { return base + hi * (T + 1) + lo; }
};

// Transform-major without padding: the index is XOR-swizzled with its own block number,
// idx ^ ((idx / T) mod T), so that both exchange access patterns (consecutive idx in
// pass 1, stride-T idx in pass 2) spread over all banks.  L * (#transforms) elements.
template <int L>
struct AddrSwizzled {
    int base;   // transform index * L
    static constexpr int T = FftShape<L>::T;
    __device__ __forceinline__ int operator()(int idx) const {
        return base + (idx ^ ((idx / T) & (T - 1)));
    }
    template <int T_>
    __device__ __forceinline__ int at(int hi, int lo) const { return base + hi * T + (lo ^ (hi & (T - 1))); }
};

// QT transforms interleaved, each with one pad element per T (index hi*T + lo sits at
// hi*(T+1) + lo): the stride-T reads of pass 2 fall on different banks even when only a
// few transforms share a warp.  (L + L/T) * QT elements.
template <int QT, int T>
struct AddrPaddedInterleaved {
    int ql;
    __device__ __forceinline__ int operator()(int idx) const { return (idx + idx / T) * QT + ql; }
    template <int T_>
    __device__ __forceinline__ int at(int hi, int lo) const { return (hi * (T + 1) + lo) * QT + ql; }
};

// QC columns per row (QC = P * QT), XOR-swizzled per row: column c of row idx sits at
// idx * QC + (c ^ (CW * key(idx))), key = (idx ^ (idx / R)) mod (R / 2), CW = 32 / R.  For
// the inner R-thread transform of fft_cyclic3 a warp touches R rows at once (consecutive
// idx in pass 1, idx strided by R in pass 2) with CW consecutive columns each; the key
// places those rows on different bank groups in both patterns (needs QT * R <= 32).
template <int QC, int R>
struct AddrInterleavedSwz {
    int c;
    static constexpr int CW = 32 / R, NPOS = R / 2;
    static_assert(R >= 1 && (R & (R - 1)) == 0 && CW * R == 32, "R a power of two <= 32");
    __device__ __forceinline__ static int key(int idx) {
        if constexpr (NPOS > 1) return (idx ^ (idx / R)) & (NPOS - 1);
        else return 0;
    }
    __device__ __forceinline__ int operator()(int idx) const { return idx * QC + (c ^ (CW * key(idx))); }
    template <int T_>
    __device__ __forceinline__ int at(int hi, int lo) const {
        const int idx = hi * T_ + lo;
        return idx * QC + (c ^ (CW * key(idx)));
    }
};

struct SyncBlock {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct SyncWarp {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
// named barrier `id` over the 128 threads of one group of four warps
struct SyncGroup128 {
    int id;
    __device__ __forceinline__ void operator()() const {
        asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory");
    }
};

// In-place L-point transform of a group of transforms whose threads run in lockstep.
//   v    thread's P points, cyclic layout in and out
//   i    thread index within its transform (0..T-1)
//   xs   shared scratch; element addresses given by addr
//   tw   pass twiddles in host_pass_twiddles layout (shared or global memory)
// sync() must make shared-memory writes of every thread of the group visible.
template <int L, bool INV, typename Addr, typename Sync>
__device__ __forceinline__ void fft_cyclic(float2 (&v)[FftShape<L>::P], int i, float2* xs,
                                           Addr addr, const float2* tw, Sync sync) {
    constexpr int P = FftShape<L>::P;
    constexpr int T = FftShape<L>::T;
    dft_reg<P, INV>(v);
    if constexpr (T > 1) {
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            float2 a = v[k1];
            if (k1 > 0) {
                const float2 w = tw[k1 * T + i];
                a = INV ? cmul_conj(a, w) : cmul(a, w);
            }
            xs[addr.template at<T>(k1, i)] = a;
            if ((k1 & 7) == 7) hoist_fence();
        }
        sync();
        constexpr int G = P / T;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            float2 w[T];
#pragma unroll
            for (int ip = 0; ip < T; ++ip) w[ip] = xs[addr.template at<T>(i + T * g, ip)];
            dft_reg<T, INV>(w);
#pragma unroll
            for (int k2 = 0; k2 < T; ++k2) v[g + G * k2] = w[k2];
        }
        sync();
    }
}

// ------------------------------------------------------------------ three-pass FFT
// L = P * T with T = P * R threads per transform (R <= P): lengths 2048 .. 32768 at P = 32.
// Pass 1: P-point DFT over u inside each thread (data x[i + T u]), twiddle w_L^{i k1}; one
// exchange hands each group of R threads one k1 (thread j plays (k1, r) = (j / R, j % R)
// and holds i = r + R u); the inner T-point DFT over i is the two-pass fft_cyclic<T> run by
// those R threads.  The result X[k1 + P k2], k2 = r + R u, sits in thread j at
// X[sigma(j) + T u], sigma(j) = (j / R) + P (j % R): cyclic in the permuted index sigma(j),
// which later stages (and an inverse transform called with i = sigma(j)) use as the
// thread's logical index.
__host__ __device__ constexpr int fft3_sigma(int j, int P, int R) { return j / R + P * (j % R); }

// Exchange placement for the pass-1 -> inner handover: element (k1, i) of transform ql at
// (k1 * (T + PAD) + j) * QT + ql.  PAD makes the reads (several k1 per warp) use both halves
// of the banks.  With R >= 8, an XOR of j with higher bits of i spreads writes whose lanes
// hold indices 32 / R apart (a transform fed in another one's output order: eight-way on
// one bank otherwise); below that j = i (two-way at R = 4 measured cheaper than the
// swizzle's per-element index arithmetic).  (P * (T + PAD) * QT elements.)
template <int QT, int T, int PAD>
struct AddrHandover {
    int ql;
    static_assert(T % 16 == 0, "the swizzle changes only the low bits of i");
    __device__ __forceinline__ int operator()(int k1, int i) const {
        // T = 512 (R = 16, one transform per warp row): lanes 32 apart, j = i ^ ((i >> 5) mod 16)
        const int j = T >= 512 ? (i ^ ((i >> 5) & 15)) : T == 256 ? (i ^ ((i >> 4) & 7)) : i;
        return (k1 * (T + PAD) + j) * QT + ql;
    }
};

// xs holds max(P (T + PAD) QT, L QT) elements; QT transforms interleaved (transform ql).
// Pass-1 twiddles w_L^{i k1} from a quarter-wave table q[k] = (cos 2 pi k / L, sin 2 pi k / L),
// k = 0 .. L/4, and the quadrant of the exponent (exact symmetry: no extra rounding).
template <int L>
struct TwiddleQuarter {
    const float2* q;
    __device__ __forceinline__ float2 operator()(int k1, int i) const {
        const int j = (k1 * i) & (L - 1);
        const int quad = j / (L / 4), r = j & (L / 4 - 1);
        const float2 b = q[r];
        const float cq = (quad & 1) ? b.y : b.x;          // cos / sin of the reduced angle,
        const float sq = (quad & 1) ? b.x : b.y;          // swapped in odd quadrants
        const float c = (quad == 1 || quad == 2) ? -cq : cq;
        const float s = (quad >= 2) ? -sq : sq;
        return make_float2(c, -s);                        // exp(-2 pi i j / L)
    }
    // Lanes read q at indices k1 * i apart: a power-of-two factor of k1 folds them onto
    // fewer banks.  fft_cyclic3 reads only odd k1 from the table and forms
    // w^{k1 i} = w^{(k1 - 1) i} w^{i} for even k1 (one more rounding, no bank conflict).
    static constexpr bool kEvenByProduct = true;
};
// ... or from a full table in host_pass_twiddles layout
struct TwiddleTable {
    static constexpr bool kEvenByProduct = false;
    const float2* t;
    int T;
    __device__ __forceinline__ float2 operator()(int k1, int i) const { return t[k1 * T + i]; }
};

// i_in: the thread's input index (it holds x[i_in + T u]); i_grp: the index whose group it
// joins for the inner transform (k1 = i_grp / R, r = i_grp % R); the output is
// X[sigma(i_grp) + T u].  i_in = i_grp = i is the plain transform.  A transform whose input
// arrives in another transform's output order calls it with i_in = sigma(i), i_grp = i: no
// reordering exchange, the lanes of a warp then read their pass-1 twiddles 32 / R index
// steps apart, so PERM forms them by the recurrence w^{k1 i} = w^{(k1 - 1) i} w^{i} with a
// table read every eight steps (at most seven extra roundings).
template <int L, bool INV, int QT, int PAD, bool PERM = false, typename Tw1, typename Sync>
__device__ __forceinline__ void fft_cyclic3(float2 (&v)[32], int i_in, int i_grp, int ql, float2* xs,
                                            Tw1 tw1, const float2* tw_in, Sync sync) {
    constexpr int P = 32;
    constexpr int T = L / P;
    constexpr int R = T / P;
    static_assert(T % P == 0 && R >= 2 && R <= P, "three-pass FFT: 2048 <= L <= 32768");
    const AddrHandover<QT, T, PAD> hand{ql};
    dft_reg<P, INV>(v);
    float2 w_one = make_float2(1.f, 0.f), w_prev = w_one;
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
        float2 a = v[k1];
        if (k1 > 0) {
            float2 w;
            if constexpr (PERM) {
                w = (k1 == 1 || (k1 & 7) == 0) ? tw1(k1, i_in) : cmul(w_prev, w_one);
            } else if constexpr (Tw1::kEvenByProduct) {
                w = (k1 & 1) ? tw1(k1, i_in) : cmul(w_prev, w_one);
            } else {
                w = tw1(k1, i_in);
            }
            if (k1 == 1) w_one = w;
            w_prev = w;
            a = INV ? cmul_conj(a, w) : cmul(a, w);
        }
        xs[hand(k1, i_in)] = a;
        if ((k1 & 7) == 7) hoist_fence();
    }
    sync();
    const int k1 = i_grp / R, r = i_grp % R;
#pragma unroll
    for (int u = 0; u < P; ++u) v[u] = xs[hand(k1, r + R * u)];
    sync();                                   // handover read: the region takes the inner exchange
    static_assert(QT * R <= 32, "a warp covers whole groups of R threads");
    const AddrInterleavedSwz<P * QT, R> inner{k1 * QT + ql};
    fft_cyclic<T, INV>(v, r, xs, inner, tw_in, sync);
}

}  // namespace ddm
