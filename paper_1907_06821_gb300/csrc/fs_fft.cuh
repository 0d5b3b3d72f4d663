// Line FFTs of the H application: in-register DFTs and in-place passes over
// lines held in shared memory.
//
// A line of length L = A * B is transformed in two passes, each thread
// holding one short DFT in registers (four-step Cooley-Tukey):
//
//   inverse (sign +), natural input x[n], n = n2 + B n1:
//     pass 1 ("stride"):  thread n2 takes x[n2 + B j] (j < A), DFT_A over j,
//                         multiplies output k1 by w_L^{n2 k1}, stores it at
//                         position n2 + B k1;
//     pass 2 ("block"):   thread k1 takes positions B k1 + j (j < B), DFT_B,
//                         stores output k2 at position B k1 + k2, which then
//                         holds X[k1 + A k2]   (the "permuted" layout).
//   forward (sign -), permuted input, natural output:
//     pass 1 ("block"):   thread k1 takes positions B k1 + j, DFT_B, multiplies
//                         output m2 by w_L^{-k1 m2}, stores it in place;
//     pass 2 ("stride"):  thread m2 takes positions m2 + B j, DFT_A, stores
//                         output m1 at position m2 + B m1 = natural index.
//
// Every pass reads and writes the same positions from the same thread, so it
// runs in place; threads only synchronise between passes.  The inverse
// transform leaves the permuted layout (position B k1 + k2 holds the value of
// index k1 + A k2) and the forward transform consumes it, so no reordering
// pass exists anywhere.  The kernels give the lanes of a warp the same role
// in consecutive lines, so with an odd line pitch both passes are free of
// shared-memory bank conflicts.  (LineGeo still allows a padded block pitch.)
//
// The in-register DFT of length N (natural order in and out) is decomposed at
// compile time into radix-2/3/4/5 butterflies with twiddles taken from the
// line's table tw[p] = exp(-2 pi i p / L), which every length here divides.
#pragma once

#include "fs_common.cuh"

// ------------------------------------------------------------------ butterflies
// out[k] = sum_r v[r] exp(s * 2 pi i r k / R), s = +1 (inverse) or -1 (forward)
template <typename T2> __device__ __forceinline__ T2 mul_si(T2 a, int s) {  // a * (s i)
    return s > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);
}

template <typename T2, int R> struct Bfly;

template <typename T2> struct Bfly<T2, 2> {
    __device__ __forceinline__ static void run(T2* v, int) {
        T2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <typename T2> struct Bfly<T2, 4> {
    __device__ __forceinline__ static void run(T2* v, int s) {
        T2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        T2 t2 = cadd(v[1], v[3]), t3 = mul_si(csub(v[1], v[3]), s);
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

template <typename T2> struct Bfly<T2, 3> {
    __device__ __forceinline__ static void run(T2* v, int s) {
        using R = typename real_of<T2>::t;
        const R h = (R)0.86602540378443864676;  // sqrt(3)/2
        T2 t = cadd(v[1], v[2]);
        T2 d = mul_si(cscale(csub(v[1], v[2]), h), s);
        T2 a = csub(v[0], cscale(t, (R)0.5));
        v[0] = cadd(v[0], t);
        v[1] = cadd(a, d);
        v[2] = csub(a, d);
    }
};

template <typename T2> struct Bfly<T2, 5> {
    __device__ __forceinline__ static void run(T2* v, int s) {
        using R = typename real_of<T2>::t;
        // cos and sin of 2 pi / 5 and 4 pi / 5
        const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;
        const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;
        T2 a14 = cadd(v[1], v[4]), d14 = csub(v[1], v[4]);
        T2 a23 = cadd(v[2], v[3]), d23 = csub(v[2], v[3]);
        T2 r1 = cadd(v[0], cadd(cscale(a14, c1), cscale(a23, c2)));
        T2 r2 = cadd(v[0], cadd(cscale(a14, c2), cscale(a23, c1)));
        T2 i1 = mul_si(cadd(cscale(d14, s1), cscale(d23, s2)), s);
        T2 i2 = mul_si(csub(cscale(d14, s2), cscale(d23, s1)), s);
        v[0] = cadd(v[0], cadd(a14, a23));
        v[1] = cadd(r1, i1);
        v[4] = csub(r1, i1);
        v[2] = cadd(r2, i2);
        v[3] = csub(r2, i2);
    }
};

// w = exp(S 2 pi i idx / L) from the table of exp(-2 pi i p / L)
template <int S, typename T2> __device__ __forceinline__ T2 twid(const T2* tw, int idx) {
    T2 w = tw[idx];
    if (S > 0) w.y = -w.y;
    return w;
}

// first radix of an in-register DFT of length n (n itself for the base cases)
__host__ __device__ constexpr int rdft_factor(int n) {
    return (n % 4 == 0 && n != 4) ? 4 : (n % 3 == 0 && n != 3) ? 3 : (n % 2 == 0 && n != 2) ? 2 : (n % 5 == 0 && n != 5) ? 5 : n;
}

// In-register DFT of length N, natural order in and out.  st = L / N: the
// twiddle w_N^e is tw[e * st].
template <int N> struct RDft {
    template <int S, typename T2> __device__ __forceinline__ static void run(T2* v, const T2* tw, int st) {
        constexpr int F = rdft_factor(N), M = N / F;
        T2 out[N];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            T2 u[F];
#pragma unroll
            for (int f = 0; f < F; ++f) u[f] = v[m + M * f];
            RDft<F>::template run<S>(u, tw, st * M);
#pragma unroll
            for (int k1 = 1; k1 < F; ++k1) {
                const int e = (m * k1) % N;
                if (e) u[k1] = cmul(u[k1], twid<S>(tw, e * st));
            }
#pragma unroll
            for (int k1 = 0; k1 < F; ++k1) v[m + M * k1] = u[k1];
        }
#pragma unroll
        for (int k1 = 0; k1 < F; ++k1) {
            T2 t[M];
#pragma unroll
            for (int m = 0; m < M; ++m) t[m] = v[m + M * k1];
            RDft<M>::template run<S>(t, tw, st * F);
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) out[k1 + F * k2] = t[k2];
        }
#pragma unroll
        for (int n = 0; n < N; ++n) v[n] = out[n];
    }
};
template <> struct RDft<1> {
    template <int S, typename T2> __device__ __forceinline__ static void run(T2*, const T2*, int) {}
};
#define FS_RDFT_BASE(R)                                                                                      \
    template <> struct RDft<R> {                                                                             \
        template <int S, typename T2> __device__ __forceinline__ static void run(T2* v, const T2*, int) {    \
            Bfly<T2, R>::run(v, S);                                                                          \
        }                                                                                                    \
    };
FS_RDFT_BASE(2)
FS_RDFT_BASE(3)
FS_RDFT_BASE(4)
FS_RDFT_BASE(5)
#undef FS_RDFT_BASE


// Stride pass on the line at `line`: role r < B, DFT_A over positions r + B j.
// TW multiplies output k1 by w_L^{S r k1} (inverse pass 1).
template <int A, int S, bool TW, typename T2>
__device__ __forceinline__ void pass_stride(T2* line, const LineGeo& g, int r, const T2* tw) {
    T2 v[A];
#pragma unroll
    for (int j = 0; j < A; ++j) v[j] = line[(r + g.Bp * j) * g.es];
    RDft<A>::template run<S>(v, tw, g.B);
    if (TW) {
#pragma unroll
        for (int k = 1; k < A; ++k)
            if (r) v[k] = cmul(v[k], twid<S>(tw, r * k));
    }
#pragma unroll
    for (int j = 0; j < A; ++j) line[(r + g.Bp * j) * g.es] = v[j];
}

// Block pass: role k1 < A, DFT_B over positions B k1 + j.  TW multiplies
// output m2 by w_L^{S k1 m2} (forward pass 1).
template <int B, int S, bool TW, typename T2>
__device__ __forceinline__ void pass_block(T2* line, const LineGeo& g, int k1, const T2* tw) {
    T2 v[B];
    const int base = g.Bp * k1;
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = line[(base + j) * g.es];
    RDft<B>::template run<S>(v, tw, g.A);
    if (TW) {
#pragma unroll
        for (int m = 1; m < B; ++m)
            if (k1) v[m] = cmul(v[m], twid<S>(tw, k1 * m));
    }
#pragma unroll
    for (int j = 0; j < B; ++j) line[(base + j) * g.es] = v[j];
}

// The register DFT sizes the passes are instantiated for: the small set keeps
// the register count of a kernel low; the large set adds 16 and 27 (for
// lengths such as 432 = 27 x 16).
#define FS_FFT_SIZES_S(X) X(1) X(2) X(3) X(4) X(5) X(6) X(8) X(9) X(10) X(12)
#define FS_FFT_SIZES_L(X) FS_FFT_SIZES_S(X) X(16) X(27)

__host__ __device__ constexpr bool fft_size_small(int n) {
    return n == 1 || n == 2 || n == 3 || n == 4 || n == 5 || n == 6 || n == 8 || n == 9 || n == 10 || n == 12;
}
__host__ __device__ constexpr bool fft_size_ok(int n) { return fft_size_small(n) || n == 16 || n == 27; }

template <int S, bool TW, bool BIG, typename T2>
__device__ __forceinline__ void stride_pass(T2* line, const LineGeo& g, int r, const T2* tw) {
#define FS_CASE(n) \
    case n: pass_stride<n, S, TW>(line, g, r, tw); break;
    if (BIG) {
        switch (g.A) { FS_FFT_SIZES_L(FS_CASE) default: break; }
    } else {
        switch (g.A) { FS_FFT_SIZES_S(FS_CASE) default: break; }
    }
#undef FS_CASE
}

template <int S, bool TW, bool BIG, typename T2>
__device__ __forceinline__ void block_pass(T2* line, const LineGeo& g, int k1, const T2* tw) {
#define FS_CASE(n) \
    case n: pass_block<n, S, TW>(line, g, k1, tw); break;
    if (BIG) {
        switch (g.B) { FS_FFT_SIZES_L(FS_CASE) default: break; }
    } else {
        switch (g.B) { FS_FFT_SIZES_S(FS_CASE) default: break; }
    }
#undef FS_CASE
}

// Logical position p of a padded line -> slot.
__device__ __forceinline__ int line_slot(const LineGeo& g, int p) { return geo_slot(g, p); }
