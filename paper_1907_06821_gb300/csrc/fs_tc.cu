// Complex GEMMs of the FP32 stage on the 5th-generation tensor cores.
//
// tcgen05.mma kind::tf32 with FP32 accumulators in tensor memory.  Each FP32
// operand x is split into x_hi = tf32(x) and x_lo = tf32(x - x_hi); the
// product a.b is taken as a_hi.b_hi + a_hi.b_lo + a_lo.b_hi (three MMAs), which
// keeps about 21 bits of the FP32 product (the split method of Ootomo and
// Yokota, 2022, with TF32 in place of FP16).
//
// Complex arithmetic is carried by real GEMMs on interleaved (re, im) data:
//   Gram form  C(i,j) = sum_k conj(a_ik) b_jk
//     UMMA A = rows a_i as 2K reals; UMMA B = rows (b_j) and (i b_j)^* rotated:
//     row 2j = (re, im) pairs of b_j, row 2j+1 = (im, -re) pairs, so that
//     D[i][2j] = Re C, D[i][2j+1] = Im C.
//   Apply form C[i][g] = sum_k A(i,k) B[k][g]
//     UMMA A = rows j' = 2g + c of the 2x2 real blocks [[re, -im], [im, re]]
//     of B[k][g]; UMMA B = rows i of A(i,k) as (re, im) pairs; D[j'][i] is
//     component c of C[i][g].
// Operands are staged by the thread block: global loads run two k-blocks
// ahead into registers, then each value is split and stored to shared memory
// in the canonical K-major no-swizzle layout (two stages); one thread issues
// the MMAs of a stage and commits them to that stage's mbarrier.
// Every mbarrier wait is bounded; on expiry the kernel raises the context's
// error flag and stops issuing work.
#include "fs_common.cuh"

#include <algorithm>
#include <mutex>

namespace {

constexpr int BK = 32;            // FP32 k elements per stage (128 bytes per row)
constexpr int TM = 128;           // UMMA M (rows of the accumulator = TMEM lanes)
constexpr int TN_MAX = 256;       // UMMA N maximum
constexpr int THREADS = 256;
constexpr int A_BYTES = TM * BK * 4;          // one split of the A tile
constexpr int B_BYTES = TN_MAX * BK * 4;      // one split of the B tile
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 64;
constexpr long long WAIT_LIMIT = 1ll << 28;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// byte offset of (row, k) in a K-major tile: 8-row x 16-byte core matrices, K fastest
__device__ __forceinline__ uint32_t kmaj(int row, int k) {
    return (uint32_t)((((row >> 3) * (BK / 4) + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2));
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;              // leading byte offset: next core matrix along K
    d |= (uint64_t)(((BK / 4) * 128) >> 4) << 32;  // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                         // descriptor version
    return d;                                       // base offset 0, no swizzle
}

__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void put2(unsigned char* hi, unsigned char* lo, uint32_t off, float a, float b) {
    float ah = tf32_rna(a), bh = tf32_rna(b);
    *reinterpret_cast<float2*>(hi + off) = make_float2(ah, bh);
    *reinterpret_cast<float2*>(lo + off) = make_float2(tf32_rna(a - ah), tf32_rna(b - bh));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
}

// bounded wait on a phase parity; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    uint32_t a = smem_u32(bar);
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared machinery: TMEM allocation, the k loop and the drain.
struct TcCtl {
    uint64_t* bar;       // [2] one per stage: MMAs reading the stage have completed
    uint32_t* tslot;     // TMEM address written by tcgen05.alloc
    unsigned char* st[2];
};

__device__ __forceinline__ TcCtl tc_setup(unsigned char* smem) {
    TcCtl t;
    t.st[0] = smem;
    t.st[1] = smem + STAGE_BYTES;
    t.bar = reinterpret_cast<uint64_t*>(smem + 2 * STAGE_BYTES);
    t.tslot = reinterpret_cast<uint32_t*>(smem + 2 * STAGE_BYTES + 32);
    if (threadIdx.x == 0) {
        mbar_init(&t.bar[0]);
        mbar_init(&t.bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(t.tslot)),
                     "r"(TN_MAX));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return t;
}

__device__ __forceinline__ void tc_teardown(const TcCtl& t) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*t.tslot), "r"(TN_MAX));
    }
}

// issue the 3 x (BK/8) MMAs of one stage
__device__ __forceinline__ void tc_issue(const TcCtl& t, int s, uint32_t tmem, uint32_t idesc, bool first) {
    uint32_t base = smem_u32(t.st[s]);
    uint32_t ahi = base, alo = base + A_BYTES, bhi = base + 2 * A_BYTES, blo = bhi + B_BYTES;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int ks = 0; ks < BK / 8; ++ks) {
        uint32_t o = ks * 256;  // two 16-byte core matrices per K = 8 step
        mma_tf32(tmem, sdesc(ahi + o), sdesc(bhi + o), idesc, (first && ks == 0) ? 0u : 1u);
        mma_tf32(tmem, sdesc(ahi + o), sdesc(blo + o), idesc, 1u);
        mma_tf32(tmem, sdesc(alo + o), sdesc(bhi + o), idesc, 1u);
    }
    mma_commit(&t.bar[s]);
}

// split a 16-byte chunk into hi/lo and store both at byte offset off of (hi, lo)
__device__ __forceinline__ void put4(unsigned char* hi, unsigned char* lo, uint32_t off, float4 v) {
    float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
    float4 l = make_float4(tf32_rna(v.x - h.x), tf32_rna(v.y - h.y), tf32_rna(v.z - h.z), tf32_rna(v.w - h.w));
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) = l;
}

// two consecutive complex values of a row (zeros past kend); rows are only 8-byte aligned
__device__ __forceinline__ float4 load2c(const float2* row, int k, int kend) {
    float2 a = make_float2(0.f, 0.f), b = a;
    if (k < kend) a = __ldg(row + k);
    if (k + 1 < kend) b = __ldg(row + k + 1);
    return make_float4(a.x, a.y, b.x, b.y);
}

// The accumulation inside tensor memory loses accuracy with the length of
// the chain (measured: the error of an H application grows about linearly
// with the number of k-blocks accumulated in place).  Every DRAIN k-blocks
// the partial tile is read out and added to FP32 registers with ordinary
// round-to-nearest adds, and the next MMA starts a fresh chain.
constexpr int DRAIN = 8;

// Per thread: TMEM lanes 32 (w & 3) .. +31, columns 128 (w >> 2) .. +127.
struct Acc {
    float v[4][32];
};

__device__ __forceinline__ void drain_add(uint32_t tmem, int ncols, Acc& a) {
    const int w = threadIdx.x >> 5;
    const int c_base = 128 * (w >> 2);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c0 = c_base + 32 * j;
        if (c0 < ncols) {  // warp-uniform
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * (w & 3)) << 16) + c0, v);
#pragma unroll
            for (int q = 0; q < 32; ++q) a.v[j][q] += v[q];
        }
    }
}

// One k-block: wait for the stage, store the registers loaded earlier, start
// the loads two k-blocks ahead, then issue the stage's MMAs.
template <class P>
__device__ __forceinline__ bool tc_step(const TcCtl& t, int kb, int nkb, uint32_t tmem, uint32_t idesc, P& p,
                                        typename P::Regs& r) {
    const int s = kb & 1;
    bool ok = true;
    if (kb >= 2) ok = mbar_wait(&t.bar[s], ((kb - 2) >> 1) & 1);
    if (!__syncthreads_and(ok)) {
        // give the MMAs already issued one more bounded chance to finish
        // before the caller releases tensor memory
        mbar_wait(&t.bar[(kb - 1) & 1], ((kb - 1) >> 1) & 1);
        return false;
    }
    p.store(r, t.st[s], t.st[s] + A_BYTES, t.st[s] + 2 * A_BYTES, t.st[s] + 2 * A_BYTES + B_BYTES);
    if (kb + 2 < nkb) p.load(r, kb + 2);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) tc_issue(t, s, tmem, idesc, kb % DRAIN == 0);
    return true;
}

// Wait for the MMAs of k-block kb, add the tile to the registers, and make
// sure every thread has read tensor memory before the next chain overwrites it.
__device__ __forceinline__ bool tc_drain(const TcCtl& t, int kb, uint32_t tmem, int ncols, Acc& a) {
    bool ok = mbar_wait(&t.bar[kb & 1], (kb >> 1) & 1);
    if (!__syncthreads_and(ok)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    drain_add(tmem, ncols, a);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    return true;
}

template <class P>
__device__ bool tc_run(const TcCtl& t, int nkb, uint32_t tmem, uint32_t idesc, int ncols, P& p, Acc& a) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 32; ++q) a.v[j][q] = 0.f;
    typename P::Regs r0, r1;
    if (nkb > 0) p.load(r0, 0);
    if (nkb > 1) p.load(r1, 1);
    for (int kb = 0; kb < nkb; kb += 2) {
        if (!tc_step(t, kb, nkb, tmem, idesc, p, r0)) return false;
        if ((kb % DRAIN == DRAIN - 1 || kb == nkb - 1) && !tc_drain(t, kb, tmem, ncols, a)) return false;
        if (kb + 1 < nkb) {
            if (!tc_step(t, kb + 1, nkb, tmem, idesc, p, r1)) return false;
            if (((kb + 1) % DRAIN == DRAIN - 1 || kb + 1 == nkb - 1) && !tc_drain(t, kb + 1, tmem, ncols, a))
                return false;
        }
    }
    return true;
}

// ---------------------------------------------------------------- Gram form
// part[z][i][j] (float2) = sum over this split's k of conj(A[i][k]) B[j][k]
struct GramP {
    const float2* A;
    long lda;
    const int* amap;
    const float2* B;
    long ldb;
    const int* bmap;
    int M, N, i0, j0, nj, kbeg, kend;
    struct Regs {
        float4 a[4], b[4];
    };
    // A task t in [0, 1024): row (t>>6)*8 + (t&7), chunk (t>>3)&7 -> smem byte 16 t
    // B task t in [0, 1024): source row (t>>5)*4 + (t&3), chunk (t>>2)&7
    __device__ __forceinline__ void load(Regs& r, int kb) const {
        const int kc0 = kbeg + kb * (BK / 2);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = threadIdx.x + THREADS * q;
            const int row = ((t >> 6) << 3) + (t & 7), ch = (t >> 3) & 7;
            const int i = i0 + row;
            r.a[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < M) r.a[q] = load2c(A + (amap ? (long)amap[i] : (long)i) * lda, kc0 + 2 * ch, kend);
            const int jj = ((t >> 5) << 2) + (t & 3), chb = (t >> 2) & 7;
            r.b[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (jj < nj) {
                const int j = j0 + jj;
                r.b[q] = load2c(B + (bmap ? (long)bmap[j] : (long)j) * ldb, kc0 + 2 * chb, kend);
            }
        }
    }
    __device__ __forceinline__ void store(const Regs& r, unsigned char* ahi, unsigned char* alo, unsigned char* bhi,
                                          unsigned char* blo) const {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = threadIdx.x + THREADS * q;
            put4(ahi, alo, 16u * t, r.a[q]);
            const int jj = ((t >> 5) << 2) + (t & 3), chb = (t >> 2) & 7;
            const float4 v = r.b[q];
            put4(bhi, blo, kmaj(2 * jj, 4 * chb), v);
            put4(bhi, blo, kmaj(2 * jj + 1, 4 * chb), make_float4(v.y, -v.x, v.w, -v.z));
        }
    }
};

__global__ void __launch_bounds__(THREADS)
tc_gram_kernel(int M, int N, int K, const float2* __restrict__ A, long lda, const int* __restrict__ amap,
               const float2* __restrict__ B, long ldb, const int* __restrict__ bmap, float2* __restrict__ part,
               int kchunk, int* errflag) {
    extern __shared__ __align__(1024) unsigned char smem[];
    TcCtl t = tc_setup(smem);
    const uint32_t tmem = *t.tslot;
    GramP p;
    p.A = A;
    p.lda = lda;
    p.amap = amap;
    p.B = B;
    p.ldb = ldb;
    p.bmap = bmap;
    p.M = M;
    p.N = N;
    p.i0 = blockIdx.x * TM;
    p.j0 = blockIdx.y * (TN_MAX / 2);
    p.nj = min(TN_MAX / 2, N - p.j0);
    p.kbeg = blockIdx.z * kchunk;
    p.kend = min(K, p.kbeg + kchunk);
    const int ncols = ((2 * p.nj + 15) / 16) * 16;  // UMMA N
    const int nkb = (2 * (p.kend - p.kbeg) + BK - 1) / BK;
    Acc acc;
    bool ok = tc_run(t, nkb, tmem, idesc_tf32(TM, ncols), ncols, p, acc);
    if (ok) {
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int i = p.i0 + 32 * (w & 3) + lane;
        float2* out = part + ((long)blockIdx.z * M + i) * N + p.j0;
        if (i < M) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c0 = 128 * (w >> 2) + 32 * j;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    int jj = c0 / 2 + q;
                    if (jj < p.nj) out[jj] = make_float2(acc.v[j][2 * q], acc.v[j][2 * q + 1]);
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(errflag, 1);
    }
    tc_teardown(t);
}

__global__ void tc_gram_reduce_kernel(int M, int N, int splits, const float2* __restrict__ part, double2* C, long ci,
                                      long cj, double alpha, double beta) {
    long total = (long)M * N;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        double sx = 0, sy = 0;
        for (int s = 0; s < splits; ++s) {
            float2 v = part[(long)s * total + t];
            sx += v.x;
            sy += v.y;
        }
        long i = t / N, j = t - i * N;
        double2* dst = C + i * ci + j * cj;
        double2 o = make_double2(alpha * sx, alpha * sy);
        if (beta != 0.0) {
            o.x += beta * dst->x;
            o.y += beta * dst->y;
        }
        *dst = o;
    }
}

// ---------------------------------------------------------------- apply form
// C[ic(i)][g] = alpha sum_k coef[i][k] B[ib(k)][g] + beta D[ic(i)][g], coef compact [M][K] float2
struct NnP {
    const float2* B;
    long ldb;
    const int* bmap;
    const float2* coef;
    int ldk;
    int N, K, g0, i0, ni, ncols;
    struct Regs {
        float4 v[2], c[8];
    };
    // UMMA A task t in [0, 512): plane wave g0 + (t & 63), complex k pair t >> 6
    // UMMA B task t in [0, 2048): coefficient row (t>>6)*8 + (t&7), chunk (t>>3)&7 -> smem byte 16 t
    __device__ __forceinline__ void load(Regs& r, int kb) const {
        const int kc0 = kb * (BK / 2);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int t = threadIdx.x + THREADS * q;
            const int g = g0 + (t & 63), k = kc0 + 2 * (t >> 6);
            float2 a = make_float2(0.f, 0.f), b = a;
            if (g < N) {
                if (k < K) a = __ldg(B + (bmap ? (long)bmap[k] : (long)k) * ldb + g);
                if (k + 1 < K) b = __ldg(B + (bmap ? (long)bmap[k + 1] : (long)(k + 1)) * ldb + g);
            }
            r.v[q] = make_float4(a.x, a.y, b.x, b.y);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int t = threadIdx.x + THREADS * q;
            const int row = ((t >> 6) << 3) + (t & 7), ch = (t >> 3) & 7;
            r.c[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row < ni) r.c[q] = load2c(coef + (long)(i0 + row) * ldk, kc0 + 2 * ch, K);
        }
    }
    __device__ __forceinline__ void store(const Regs& r, unsigned char* ahi, unsigned char* alo, unsigned char* bhi,
                                          unsigned char* blo) const {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int t = threadIdx.x + THREADS * q;
            const int gg = t & 63, kp = t >> 6;
            const float4 v = r.v[q];  // (re_k, im_k, re_k+1, im_k+1)
            put4(ahi, alo, kmaj(2 * gg, 4 * kp), make_float4(v.x, -v.y, v.z, -v.w));
            put4(ahi, alo, kmaj(2 * gg + 1, 4 * kp), make_float4(v.y, v.x, v.w, v.z));
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int t = threadIdx.x + THREADS * q;
            const int row = ((t >> 6) << 3) + (t & 7);
            if (row < ncols) put4(bhi, blo, 16u * t, r.c[q]);
        }
    }
};

__global__ void __launch_bounds__(THREADS)
tc_nn_kernel(int M, int N, int K, const float2* __restrict__ coef, int ldk, const float2* __restrict__ B, long ldb,
             const int* __restrict__ bmap, float2* C, long ldc, const int* __restrict__ cmap, float alpha, float beta,
             const float2* D, long ldd, int* errflag) {
    extern __shared__ __align__(1024) unsigned char smem[];
    TcCtl t = tc_setup(smem);
    const uint32_t tmem = *t.tslot;
    NnP p;
    p.B = B;
    p.ldb = ldb;
    p.bmap = bmap;
    p.coef = coef;
    p.ldk = ldk;
    p.N = N;
    p.K = K;
    p.g0 = blockIdx.x * (TM / 2);
    p.i0 = blockIdx.y * TN_MAX;
    p.ni = min(TN_MAX, M - p.i0);
    p.ncols = ((p.ni + 15) / 16) * 16;
    const int nkb = (2 * K + BK - 1) / BK;
    Acc acc;
    bool ok = tc_run(t, nkb, tmem, idesc_tf32(TM, p.ncols), p.ncols, p, acc);
    if (ok) {
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int r = 32 * (w & 3) + lane;  // j' = 2g + c
        const int g = p.g0 + (r >> 1);
        const int comp = r & 1;
        float* Cf = reinterpret_cast<float*>(C);
        const float* Df = reinterpret_cast<const float*>(D);
        if (g < N) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c0 = 128 * (w >> 2) + 32 * j;
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    int ii = c0 + q;
                    if (ii < p.ni) {
                        long row = cmap ? (long)cmap[p.i0 + ii] : (long)(p.i0 + ii);
                        float o = alpha * acc.v[j][q];
                        if (beta != 0.f) o += beta * Df[(row * ldd + g) * 2 + comp];
                        Cf[(row * ldc + g) * 2 + comp] = o;
                    }
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(errflag, 1);
    }
    tc_teardown(t);
}

// coef[i][k] = A(i, k) as float2, compact
template <typename A2>
__global__ void pack_coef_kernel(const A2* __restrict__ A, long ai, long ak, int M, int K, float2* __restrict__ coef) {
    long total = (long)M * K;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        long i = t / K, k = t - i * K;
        A2 a = A[i * ai + k * ak];
        coef[t] = make_float2((float)a.x, (float)a.y);
    }
}

std::once_flag g_attr_once;
void set_attrs_once() {
    cudaFuncSetAttribute((const void*)tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    cudaFuncSetAttribute((const void*)tc_nn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}
void set_attrs() { std::call_once(g_attr_once, set_attrs_once); }

}  // namespace

void tc_gemm_gram(fs_ctx* c, int M, int N, int K, const float2* A, long lda, const int* amap, const float2* B,
                  long ldb, const int* bmap, double2* C, long ci, long cj, double alpha, double beta, int kid) {
    if (M <= 0 || N <= 0) return;
    set_attrs();
    ProfScope ps(c, kid, ((double)M + N) * K * sizeof(float2) + (double)M * N * sizeof(double2), 8.0 * M * N * K);
    int tm = (M + TM - 1) / TM, tn = (N + TN_MAX / 2 - 1) / (TN_MAX / 2);
    int want = std::max(1, (2 * 148 + tm * tn - 1) / (tm * tn));
    int maxs = std::max(1, K / 1024);
    int splits = std::min(want, maxs);
    int kchunk = (K + splits - 1) / splits;
    kchunk = std::min(kchunk, c->tc_gram_kchunk);
    kchunk = ((kchunk + BK / 2 - 1) / (BK / 2)) * (BK / 2);
    splits = std::max(1, (K + kchunk - 1) / kchunk);
    c->splitk.ensure((size_t)splits * M * N * sizeof(float2));
    dim3 g(tm, tn, splits);
    tc_gram_kernel<<<g, THREADS, SMEM_BYTES, c->stream>>>(M, N, K, A, lda, amap, B, ldb, bmap,
                                                          c->splitk.as<float2>(), kchunk, ctx_errflag(c));
    long total = (long)M * N;
    int rb = (int)std::min<long>(2048, (total + 255) / 256);
    tc_gram_reduce_kernel<<<rb, 256, 0, c->stream>>>(M, N, splits, c->splitk.as<float2>(), C, ci, cj, alpha, beta);
    FS_CUDA(cudaGetLastError());
}

template <typename A2>
void tc_gemm_nn(fs_ctx* c, int M, int N, int K, const A2* A, long ai, long ak, const float2* B, long ldb,
                const int* bmap, float2* C, long ldc, const int* cmap, double alpha, double beta, const float2* D,
                long ldd, int kid) {
    if (M <= 0 || N <= 0) return;
    set_attrs();
    ProfScope ps(c, kid, ((double)K + M * (beta != 0.0 ? 2.0 : 1.0)) * N * sizeof(float2) + (double)M * K * sizeof(A2),
                 8.0 * M * N * K);
    c->coefbuf.ensure((size_t)M * K * sizeof(float2));
    long total = (long)M * K;
    pack_coef_kernel<A2><<<(int)std::min<long>(1024, (total + 255) / 256), 256, 0, c->stream>>>(
        A, ai, ak, M, K, c->coefbuf.as<float2>());
    dim3 g((N + TM / 2 - 1) / (TM / 2), (M + TN_MAX - 1) / TN_MAX);
    // the tensor-memory accumulation runs over at most tc_nn_kchunk complex k
    // per launch; longer sums continue in FP32 global memory (beta = 1)
    const int kc = std::max(BK / 2, c->tc_nn_kchunk);
    for (int k0 = 0; k0 < K; k0 += kc) {
        const int kk = std::min(kc, K - k0);
        const bool first = k0 == 0;
        const int* bm = bmap ? bmap + k0 : nullptr;
        const float2* Bk = bmap ? B : B + (long)k0 * ldb;
        tc_nn_kernel<<<g, THREADS, SMEM_BYTES, c->stream>>>(
            M, N, kk, c->coefbuf.as<float2>() + k0, K, Bk, ldb, bm, C, ldc, cmap, (float)alpha,
            first ? (float)beta : 1.0f, first ? D : C, first ? ldd : ldc, ctx_errflag(c));
        FS_CUDA(cudaGetLastError());
    }
}

template void tc_gemm_nn<double2>(fs_ctx*, int, int, int, const double2*, long, long, const float2*, long, const int*,
                                  float2*, long, const int*, double, double, const float2*, long, int);
template void tc_gemm_nn<float2>(fs_ctx*, int, int, int, const float2*, long, long, const float2*, long, const int*,
                                 float2*, long, const int*, double, double, const float2*, long, int);
