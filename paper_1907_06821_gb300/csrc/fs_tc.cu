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
// Formatting kernels first write each operand to global memory as the exact
// shared-memory images the MMAs read (hi and lo splits, K-major no-swizzle
// core-matrix layout, 8 complex k per stage); the projector table is
// formatted once per context.  The GEMM kernels then only move bytes: one
// thread issues bulk asynchronous copies (cp.async.bulk) into a 4-stage ring,
// one thread issues the MMAs, and eight warps drain the accumulator.
// Every mbarrier wait is bounded; on expiry the kernel raises the context's
// error flag, waits (bounded) for its copies and MMAs in flight, releases
// tensor memory and returns.
#include "fs_beta.cuh"
#include "fs_common.cuh"

#include <algorithm>
#include <mutex>

namespace {

constexpr int TM = 128;           // UMMA M (rows of the accumulator = TMEM lanes)
constexpr int TN_MAX = 256;       // UMMA N maximum
constexpr long long WAIT_LIMIT = 1ll << 28;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
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
// with the number of k-blocks accumulated in place).  Every 128 complex k the
// partial tile is read out and added to FP32 registers with ordinary
// round-to-nearest adds, and the next MMA starts a fresh chain.
// Per thread: TMEM lanes 32 (w & 3) .. +31, columns 128 (w >> 2) .. +127.
struct Acc {
    float v[4][32];
};

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
// C[ic(i)][g] = alpha sum_k A(i,k) B[ib(k)][g] + beta D[ic(i)][g].
//
// Both operands are first written to global memory as the exact shared-memory
// images the MMAs read (TF32 hi and lo splits, K-major core-matrix layout), so
// the GEMM kernel moves them with bulk asynchronous copies and does no
// arithmetic on the way in:
//   UMMA A tile (gt, kb): rows j' = 2g + c of 64 plane waves g, the 8 complex
//     k of stage kb as 16 reals, the 2x2 real block [[re, -im], [im, re]] of
//     B[k][g] (row c = 0: (re, -im) pairs, c = 1: (im, re) pairs);
//   UMMA B tile (it, kb): rows i of the coefficients A(i, k) as (re, im) pairs.
// The projector table of the nonlocal term is formatted once per context.
// Kernel roles: warp 0 issues the bulk copies into a 4-stage ring, warp 1
// issues the MMAs (three per k-step: hi.hi, hi.lo, lo.hi), warps 2-9 drain
// the tensor-memory accumulator into FP32 registers every 128 complex k, from
// two accumulator buffers so that the MMAs never wait for the drain.
constexpr int QK = 16;                        // FP32 k per stage (8 complex k, 64 bytes per row)
constexpr int QS = 4;                         // stages in the ring
constexpr int QA_BYTES = TM * QK * 4;         // one split of the A tile (8 KB)
constexpr int QB_MAX = TN_MAX * QK * 4;       // one split of the largest B tile (16 KB)
constexpr int QSTAGE = 2 * QA_BYTES + 2 * QB_MAX;
constexpr int QDRAIN = 16;                    // stages per tensor-memory chain
constexpr int QTHREADS = 320;
constexpr int QSMEM = QS * QSTAGE + 128;
// persistent apply form: as many stages of the actual tile size as fit
constexpr int QS_MAX = 8;
constexpr int QSMEM_MAX = 232448;             // the opt-in shared memory of one block
constexpr int QCTL_BYTES = 256;               // barriers and the tensor-memory slot

__host__ __device__ __forceinline__ uint32_t kmaj16(int row, int k) {
    return (uint32_t)((((row >> 3) * (QK / 4) + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2));
}

__device__ __forceinline__ uint64_t sdesc16(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;              // leading byte offset: next core matrix along K
    d |= (uint64_t)(((QK / 4) * 128) >> 4) << 32;  // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mbar_init_n(uint64_t* bar, int n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(n));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bulk copy global -> shared (16-byte aligned, size a multiple of 16), completion on bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// UMMA A tiles of B[k][g]: one thread per (g, pair of complex k)
// (plane-wave tiles gstart/64 .. +gtiles, written from tile 0 of out)
__global__ void fmt_expand_kernel(const float2* __restrict__ B, long ldb, const int* __restrict__ bmap, int K, int N,
                                  int nkb, int gstart, int gtiles, unsigned char* __restrict__ out) {
    const long ng = (long)gtiles * 64;
    const long total = ng * nkb * 4;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int gl = (int)(t % ng);
        const int g = gstart + gl;
        const int k = 2 * (int)(t / ng);
        float2 a = make_float2(0.f, 0.f), b = a;
        if (g < N) {
            if (k < K) a = __ldg(B + (bmap ? (long)bmap[k] : (long)k) * ldb + g);
            if (k + 1 < K) b = __ldg(B + (bmap ? (long)bmap[k + 1] : (long)(k + 1)) * ldb + g);
        }
        const int kb = k >> 3, kq = k & 7, gt = gl >> 6, gg = gl & 63;
        unsigned char* tile = out + ((size_t)gt * nkb + kb) * (2 * QA_BYTES);
        put4(tile, tile + QA_BYTES, kmaj16(2 * gg, 2 * kq), make_float4(a.x, -a.y, b.x, -b.y));
        put4(tile, tile + QA_BYTES, kmaj16(2 * gg + 1, 2 * kq), make_float4(a.y, a.x, b.y, b.x));
    }
}

// UMMA B tiles of the coefficients A(i, k) = A[i ai + k ak]: one thread per (i, pair of complex k)
template <typename A2>
__global__ void fmt_coef_kernel(const A2* __restrict__ A, long ai, long ak, int M, int K, int TI, int itiles, int nkb,
                                unsigned char* __restrict__ out) {
    const long ni = (long)itiles * TI;
    const long total = ni * nkb * 4;
    const uint32_t split = (uint32_t)TI * QK * 4;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t % ni);
        const int k = 2 * (int)(t / ni);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < M) {
            if (k < K) {
                A2 a = A[i * ai + k * ak];
                v.x = (float)a.x;
                v.y = (float)a.y;
            }
            if (k + 1 < K) {
                A2 a = A[i * ai + (k + 1) * ak];
                v.z = (float)a.x;
                v.w = (float)a.y;
            }
        }
        const int kb = k >> 3, kq = k & 7, it = i / TI, ii = i - it * TI;
        unsigned char* tile = out + ((size_t)it * nkb + kb) * (2 * (size_t)split);
        put4(tile, tile + split, kmaj16(ii, 2 * kq), v);
    }
}

// Barriers and tensor memory of the bulk-fed kernels (after the QS stages in shared memory).
struct QCtl {
    uint64_t* full;   // [QS] stage loaded (bulk-copy transaction bytes)
    uint64_t* empty;  // [QS] stage consumed by the MMAs
    uint64_t* accf;   // [2] accumulator chain complete
    uint64_t* acce;   // [2] accumulator drained by the 8 drain warps
    uint32_t tmem;
};

// nst stages of sbytes each, then the barriers (nst <= QS_MAX)
__device__ __forceinline__ QCtl tcq_setup(unsigned char* smem, int nst = QS, uint32_t sbytes = QSTAGE) {
    QCtl t;
    t.full = reinterpret_cast<uint64_t*>(smem + (size_t)nst * sbytes);
    t.empty = t.full + nst;
    t.accf = t.empty + nst;
    t.acce = t.accf + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(t.acce + 2);
    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init_n(&t.full[s], 1);
            mbar_init_n(&t.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init_n(&t.accf[b], 1);
            mbar_init_n(&t.acce[b], 8);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    t.tmem = *tslot;
    return t;
}

__device__ __forceinline__ void tcq_teardown(const QCtl& t, bool ok, int* errflag) {
    if (!ok) atomicExch(errflag, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t.tmem), "r"(512));
}

// The k loop over nkb stages whose A images (2 x QA_BYTES each) start at a and
// B images (2 x bsplit each, TI rows) at b.  Warp 0 copies, warp 1 issues
// the MMAs, warps 2-9 drain; on return the drain threads hold the tile in
// acc (thread: TMEM lane 32 (warp & 3) + lane, columns 128 ((warp - 2) >> 2)
// + 32 j + e).  Returns false if a bounded wait gave up.
__device__ __forceinline__ bool tcq_pipeline(const QCtl& t, unsigned char* smem, const unsigned char* a,
                                             const unsigned char* b, int nkb, int TI, Acc& acc) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bsplit = (uint32_t)TI * QK * 4;
    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {
            int last = -1;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % QS;
                if (kb >= QS && !mbar_wait(&t.empty[s], ((kb / QS) - 1) & 1)) {
                    ok = false;
                    break;
                }
                unsigned char* st = smem + s * QSTAGE;
                mbar_expect_tx(&t.full[s], 2 * QA_BYTES + 2 * bsplit);
                bulk_g2s(st, a + (size_t)kb * (2 * QA_BYTES), 2 * QA_BYTES, &t.full[s]);
                bulk_g2s(st + 2 * QA_BYTES, b + (size_t)kb * (2 * bsplit), 2 * bsplit, &t.full[s]);
                last = kb;
            }
            // every copy issued has landed before the block can exit
            for (int kb = max(0, last - QS + 1); kb <= last; ++kb)
                if (!mbar_wait(&t.full[kb % QS], (kb / QS) & 1)) ok = false;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(TM, TI);
            int last = -1;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % QS, ch = kb / QDRAIN, buf = ch & 1;
                const bool first = kb % QDRAIN == 0;
                if (!mbar_wait(&t.full[s], (kb / QS) & 1)) {
                    ok = false;
                    break;
                }
                if (first && ch >= 2 && !mbar_wait(&t.acce[buf], ((ch >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base = smem_u32(smem + s * QSTAGE);
                const uint32_t ahi = base, alo = base + QA_BYTES, bhi = base + 2 * QA_BYTES, blo = bhi + bsplit;
                const uint32_t d = t.tmem + (uint32_t)(buf * 256);
#pragma unroll
                for (int ks = 0; ks < QK / 8; ++ks) {
                    const uint32_t o = ks * 256;
                    mma_tf32(d, sdesc16(ahi + o), sdesc16(bhi + o), idesc, (first && ks == 0) ? 0u : 1u);
                    mma_tf32(d, sdesc16(ahi + o), sdesc16(blo + o), idesc, 1u);
                    mma_tf32(d, sdesc16(alo + o), sdesc16(bhi + o), idesc, 1u);
                }
                mma_commit(&t.empty[s]);
                if (kb % QDRAIN == QDRAIN - 1 || kb == nkb - 1) mma_commit(&t.accf[buf]);
                last = kb;
            }
            // the MMAs issued have completed before tensor memory is released
            if (last >= 0 && !mbar_wait(&t.empty[last % QS], (last / QS) & 1)) ok = false;
        }
    } else {
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int nchain = (nkb + QDRAIN - 1) / QDRAIN;
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 32; ++e) acc.v[j][e] = 0.f;
        for (int ch = 0; ch < nchain; ++ch) {
            const int buf = ch & 1;
            if (!mbar_wait(&t.accf[buf], (ch >> 1) & 1)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c0 = 128 * h + 32 * j;
                if (c0 < TI) {  // warp-uniform
                    float v[32];
                    tmem_ld32(t.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * 256 + c0), v);
#pragma unroll
                    for (int e = 0; e < 32; ++e) acc.v[j][e] += v[e];
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&t.acce[buf]);
        }
    }
    return ok;
}

// Persistent apply form: each block walks the tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... (t -> coefficient tile it = t mod itiles,
// plane-wave tile gt = t / itiles, so the blocks that share a plane-wave tile
// run side by side and its images come from L2 the second time).  The copy
// and MMA threads run ahead across tile boundaries with global stage and
// chain counters, so one tile's epilogue overlaps the next tile's copies and
// MMAs; the ring holds nst stages of the tile's actual size.
__global__ void __launch_bounds__(QTHREADS, 1)
tcq_nn_kernel(int M, int N, int nkb, int TI, int itiles, int ntiles, int gt0, int nst,
              const unsigned char* __restrict__ Af, const unsigned char* __restrict__ Bf, float2* C, long ldc,
              const int* __restrict__ cmap, float alpha, float beta, const float2* D, long ldd, int* errflag) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t bsplit = (uint32_t)TI * QK * 4;
    const uint32_t sbytes = 2 * QA_BYTES + 2 * bsplit;
    const QCtl t = tcq_setup(smem, nst, sbytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {
            long long g = 0;  // stages issued by this block
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                const int it = tile % itiles, gt = tile / itiles;
                const unsigned char* a = Af + (size_t)gt * nkb * (2 * QA_BYTES);
                const unsigned char* b = Bf + (size_t)it * nkb * (2 * (size_t)bsplit);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int st = (int)(g % nst);
                    if (g >= nst && !mbar_wait(&t.empty[st], (uint32_t)((g / nst) - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    unsigned char* dst = smem + (size_t)st * sbytes;
                    mbar_expect_tx(&t.full[st], sbytes);
                    bulk_g2s(dst, a + (size_t)kb * (2 * QA_BYTES), 2 * QA_BYTES, &t.full[st]);
                    bulk_g2s(dst + 2 * QA_BYTES, b + (size_t)kb * (2 * bsplit), 2 * bsplit, &t.full[st]);
                }
            }
            // every copy issued has landed before the block can exit
            for (long long q = g > nst ? g - nst : 0; q < g; ++q)
                if (!mbar_wait(&t.full[q % nst], (uint32_t)(q / nst) & 1)) ok = false;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(TM, TI);
            long long g = 0, last = -1;
            int ch = 0;  // accumulator chains started by this block
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int st = (int)(g % nst), buf = ch & 1;
                    const bool first = kb % QDRAIN == 0;
                    if (!mbar_wait(&t.full[st], (uint32_t)(g / nst) & 1)) {
                        ok = false;
                        break;
                    }
                    if (first && ch >= 2 && !mbar_wait(&t.acce[buf], ((ch >> 1) - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t base = smem_u32(smem + (size_t)st * sbytes);
                    const uint32_t ahi = base, alo = base + QA_BYTES, bhi = base + 2 * QA_BYTES, blo = bhi + bsplit;
                    const uint32_t d = t.tmem + (uint32_t)(buf * 256);
#pragma unroll
                    for (int ks = 0; ks < QK / 8; ++ks) {
                        const uint32_t o = ks * 256;
                        mma_tf32(d, sdesc16(ahi + o), sdesc16(bhi + o), idesc, (first && ks == 0) ? 0u : 1u);
                        mma_tf32(d, sdesc16(ahi + o), sdesc16(blo + o), idesc, 1u);
                        mma_tf32(d, sdesc16(alo + o), sdesc16(bhi + o), idesc, 1u);
                    }
                    mma_commit(&t.empty[st]);
                    if (kb % QDRAIN == QDRAIN - 1 || kb == nkb - 1) {
                        mma_commit(&t.accf[buf]);
                        ++ch;
                    }
                    last = g;
                }
            }
            // the MMAs issued have completed before tensor memory is released
            if (last >= 0 && !mbar_wait(&t.empty[last % nst], (uint32_t)(last / nst) & 1)) ok = false;
        }
    } else {
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int nchain = (nkb + QDRAIN - 1) / QDRAIN;
        const int r = 32 * q + lane;  // j' = 2 g + c
        const int comp = r & 1;
        float* Cf = reinterpret_cast<float*>(C);
        const float* Df = reinterpret_cast<const float*>(D);
        int ch = 0;
        Acc acc;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int it = tile % itiles, gt = tile / itiles;
            const int i0 = it * TI, ni = min(TI, M - i0), g = (gt0 + gt) * 64 + (r >> 1);
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int e = 0; e < 32; ++e) acc.v[j][e] = 0.f;
            for (int cc = 0; cc < nchain; ++cc, ++ch) {
                const int buf = ch & 1;
                // every lane polls; the vote keeps the warp together if one gives up
                if (!__all_sync(0xffffffffu, mbar_wait(&t.accf[buf], (ch >> 1) & 1))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c0 = 128 * h + 32 * j;
                    if (c0 < TI) {  // warp-uniform
                        float v[32];
                        tmem_ld32(t.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * 256 + c0), v);
#pragma unroll
                        for (int e = 0; e < 32; ++e) acc.v[j][e] += v[e];
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&t.acce[buf]);
            }
            if (!ok) break;
            if (g < N) {
                // in groups of 8 outputs: the row indices, then the D values, then the
                // stores, so that the loads of a group are in flight together (D may be
                // C itself; each thread reads only the elements it writes)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c0 = 128 * h + 32 * j;
                    if (c0 >= ni) continue;  // warp-uniform
#pragma unroll
                    for (int e0 = 0; e0 < 32; e0 += 8) {
                        long row[8];
                        float dv[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int ii = c0 + e0 + e;
                            row[e] = ii < ni ? (cmap ? (long)__ldg(cmap + i0 + ii) : (long)(i0 + ii)) : -1;
                        }
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            dv[e] = (beta != 0.f && row[e] >= 0) ? Df[(row[e] * ldd + g) * 2 + comp] : 0.f;
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (row[e] >= 0) {
                                float o = alpha * acc.v[j][e0 + e];
                                if (beta != 0.f) o += beta * dv[e];
                                Cf[(row[e] * ldc + g) * 2 + comp] = o;
                            }
                    }
                }
            }
        }
    }
    tcq_teardown(t, ok, errflag);
}

// ---------------------------------------------------------------- bulk-fed Gram form
// part[z][i][j] (float2) = sum over the stages of split z of conj(A[ia(i)][k]) B[ib(j)][k].
// UMMA A tile (it, kb): rows a_i (128 per tile) as (re, im) pairs; UMMA B tile
// (jt, kb): rows 2j = (re, im) and 2j + 1 = (im, -re) of b_j (TJ rows = TJ/2
// vectors per tile), so that D[i][2j] = Re C and D[i][2j + 1] = Im C.
// Formatting: one warp per (8-row group, stage); lane (r = lane & 7, kc =
// lane >> 3) takes complex k = 8 kb + 2 kc, kc + 1 of row r, and the 8 lanes of
// one kc write one 128-byte core matrix.

// UMMA A images of rows a_i, stages [kb0, kb0 + nkbl) written as local stages
__global__ void fmt_rows_kernel(const float2* __restrict__ A, long lda, const int* __restrict__ amap, int M, int K,
                                int itiles, int kb0, int nkbl, unsigned char* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const long nwarp = (long)itiles * 16 * nkbl;
    for (long w = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5; w < nwarp;
         w += ((long)gridDim.x * blockDim.x) >> 5) {
        const int rg = (int)(w / nkbl), kbl = (int)(w % nkbl);
        const int r = lane & 7, kc = lane >> 3;
        const int i = rg * 8 + r;
        const int k = (kb0 + kbl) * 8 + 2 * kc;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < M) v = load2c(A + (amap ? (long)amap[i] : (long)i) * lda, k, K);
        const int it = rg >> 4, rr = ((rg & 15) << 3) + r;
        unsigned char* tile = out + ((size_t)it * nkbl + kbl) * (2 * QA_BYTES);
        put4(tile, tile + QA_BYTES, kmaj16(rr, 4 * kc), v);
    }
}

// UMMA B images of rows b_j with their rotated copies, TJ output rows per tile
__global__ void fmt_rot_kernel(const float2* __restrict__ B, long ldb, const int* __restrict__ bmap, int N, int K,
                               int TJ, int jtiles, int nkbl, unsigned char* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const long nwarp = (long)jtiles * (TJ / 8) * nkbl;
    const uint32_t split = (uint32_t)TJ * QK * 4;
    for (long w = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5; w < nwarp;
         w += ((long)gridDim.x * blockDim.x) >> 5) {
        const int og = (int)(w / nkbl), kbl = (int)(w % nkbl);
        const int r = lane & 7, kc = lane >> 3;
        const int orow = og * 8 + r;
        const int jt = orow / TJ, rr = orow - jt * TJ;
        const int j = jt * (TJ / 2) + (rr >> 1);
        const int k = kbl * 8 + 2 * kc;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < N) v = load2c(B + (bmap ? (long)bmap[j] : (long)j) * ldb, k, K);
        if (rr & 1) v = make_float4(v.y, -v.x, v.w, -v.z);
        unsigned char* tile = out + ((size_t)jt * nkbl + kbl) * (2 * (size_t)split);
        put4(tile, tile + split, kmaj16(rr, 4 * kc), v);
    }
}

// Generated projectors (no table): the Gram-form A images of rows beta_p, and
// the apply-form A tiles of beta_k(q_g), in the layout fmt_rows_kernel and
// fmt_expand_kernel write from a stored FP32 table (values formed in FP32).
__global__ void fmt_beta_rows_kernel(BetaGen Bg, int M, int K, int itiles, int kb0, int nkbl,
                                     unsigned char* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const long nwarp = (long)itiles * 16 * nkbl;
    for (long w = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5; w < nwarp;
         w += ((long)gridDim.x * blockDim.x) >> 5) {
        const int rg = (int)(w / nkbl), kbl = (int)(w % nkbl);
        const int r = lane & 7, kc = lane >> 3;
        const int i = rg * 8 + r;
        const int k = (kb0 + kbl) * 8 + 2 * kc;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < M) {
            if (k < K) {
                const float2 a = beta_value32(Bg, i, k);
                v.x = a.x;
                v.y = a.y;
            }
            if (k + 1 < K) {
                const float2 a = beta_value32(Bg, i, k + 1);
                v.z = a.x;
                v.w = a.y;
            }
        }
        const int it = rg >> 4, rr = ((rg & 15) << 3) + r;
        unsigned char* tile = out + ((size_t)it * nkbl + kbl) * (2 * QA_BYTES);
        put4(tile, tile + QA_BYTES, kmaj16(rr, 4 * kc), v);
    }
}

__global__ void fmt_beta_expand_kernel(BetaGen Bg, int K, int N, int nkb, int gstart, int gtiles,
                                       unsigned char* __restrict__ out) {
    const long ng = (long)gtiles * 64;
    const long total = ng * nkb * 4;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int gl = (int)(t % ng);
        const int g = gstart + gl;
        const int k = 2 * (int)(t / ng);
        float2 a = make_float2(0.f, 0.f), b = a;
        if (g < N) {
            if (k < K) a = beta_value32(Bg, k, g);
            if (k + 1 < K) b = beta_value32(Bg, k + 1, g);
        }
        const int kb = k >> 3, kq = k & 7, gt = gl >> 6, gg = gl & 63;
        unsigned char* tile = out + ((size_t)gt * nkb + kb) * (2 * QA_BYTES);
        put4(tile, tile + QA_BYTES, kmaj16(2 * gg, 2 * kq), make_float4(a.x, -a.y, b.x, -b.y));
        put4(tile, tile + QA_BYTES, kmaj16(2 * gg + 1, 2 * kq), make_float4(a.y, a.x, b.y, b.x));
    }
}

// grid (itiles, jtiles, splits): split z takes local stages [z kbs, min(nkbl, (z + 1) kbs)) of the
// chunk; A images of row tile it start at Af + it * astride stages (+ akb0 stages), B images at
// Bf + jt * nkbl stages; partial sums go to part[(z0 + z) M N + i N + j].
__global__ void __launch_bounds__(QTHREADS, 1)
tcq_gram_kernel(int M, int N, int TJ, int nkbl, int kbs, const unsigned char* __restrict__ Af, long astride,
                long akb0, const unsigned char* __restrict__ Bf, float2* __restrict__ part, int z0, int* errflag) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const QCtl t = tcq_setup(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it = blockIdx.x, jt = blockIdx.y, z = blockIdx.z;
    const int kb0 = z * kbs, nk = min(nkbl, kb0 + kbs) - kb0;
    const int j0 = jt * (TJ / 2), nj = min(TJ / 2, N - j0);
    Acc acc;
    const bool ok = tcq_pipeline(t, smem, Af + ((size_t)it * astride + akb0 + kb0) * (2 * QA_BYTES),
                                 Bf + ((size_t)jt * nkbl + kb0) * (2 * (size_t)TJ * QK * 4), nk, TJ, acc);
    if (ok && warp >= 2) {
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int i = it * TM + 32 * q + lane;
        if (i < M) {
            float2* out = part + ((long)(z0 + z) * M + i) * N + j0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c0 = 128 * h + 32 * j;
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int jj = c0 / 2 + e;
                    if (jj < nj) out[jj] = make_float2(acc.v[j][2 * e], acc.v[j][2 * e + 1]);
                }
            }
        }
    }
    tcq_teardown(t, ok, errflag);
}

// The bounded wait of the pipelines, on a barrier that nothing completes: it
// polls `limit` times, gives up and raises the context's error flag.
__global__ void wait_selftest_kernel(long long limit, int* errflag) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init_n(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t a = smem_u32(&bar);
        bool ok = false;
        for (long long it = 0; it < limit && !ok; ++it) {
            uint32_t r;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(r)
                : "r"(a), "r"(0u)
                : "memory");
            ok = r != 0;
        }
        if (!ok) atomicExch(errflag, 1);
    }
}

std::once_flag g_attr_once;
void set_attrs_once() {
    cudaFuncSetAttribute((const void*)tcq_nn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, QSMEM_MAX);
    cudaFuncSetAttribute((const void*)tcq_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, QSMEM);
}
void set_attrs() { std::call_once(g_attr_once, set_attrs_once); }

}  // namespace

void tc_gemm_gram(fs_ctx* c, int M, int N, int K, const float2* A, long lda, const int* amap, const float2* B,
                  long ldb, const int* bmap, double2* C, long ci, long cj, double alpha, double beta, int kid,
                  const BetaGen* gen) {
    if (M <= 0 || N <= 0) return;
    set_attrs();
    ProfScope ps(c, kid, ((double)M + N) * K * sizeof(float2) + (double)M * N * sizeof(double2), 8.0 * M * N * K);
    const int nkb = std::max(1, (K + 7) / 8);
    const int itiles = (M + TM - 1) / TM;
    const int jtiles = (N + TN_MAX / 2 - 1) / (TN_MAX / 2);
    const int TJ = ((2 * ((N + jtiles - 1) / jtiles)) + 15) / 16 * 16;  // UMMA N, balanced over the tiles
    const size_t a_stage = (size_t)2 * QA_BYTES;                        // A images of one row tile, one stage
    const size_t b_stage = (size_t)2 * TJ * QK * 4;
    auto rows = [&](const unsigned char* dst, int kb0, int nkbl) {
        const long thr = (long)itiles * 16 * nkbl * 32;
        const int nbk = (int)std::min<long>(152 * 16, (thr + 255) / 256);
        if (gen)
            fmt_beta_rows_kernel<<<nbk, 256, 0, c->stream>>>(*gen, M, K, itiles, kb0, nkbl, (unsigned char*)dst);
        else
            fmt_rows_kernel<<<nbk, 256, 0, c->stream>>>(A, lda, amap, M, K, itiles, kb0, nkbl, (unsigned char*)dst);
    };
    bool table = !gen && A == c->beta32.as<float2>() && amap == nullptr && M == c->nptot && K == c->npw;
    if (table && !c->beta32_gfmt.p && (size_t)itiles * nkb * a_stage <= FS_TABLE_FMT_MAX_BYTES) {
        c->beta32_gfmt.alloc((size_t)itiles * nkb * a_stage);
        rows(c->beta32_gfmt.as<unsigned char>(), 0, nkb);
    }
    table = table && c->beta32_gfmt.p != nullptr;
    // stages per chunk of per-call images
    const size_t per_stage = (table ? 0 : itiles * a_stage) + jtiles * b_stage;
    const int kchunk = (int)std::max<size_t>(16, std::min<size_t>(nkb, FS_FMT_CHUNK_BYTES / per_stage));
    const int ntile = itiles * jtiles;
    std::vector<int> zs;
    int ztot = 0;
    for (int kc0 = 0; kc0 < nkb; kc0 += kchunk) {
        const int nkbl = std::min(kchunk, nkb - kc0);
        const int want = std::max(1, (2 * 152 + ntile - 1) / ntile);
        int splits = std::max(1, std::min(want, nkbl / (2 * QDRAIN)));
        const int kbs = (nkbl + splits - 1) / splits;
        splits = (nkbl + kbs - 1) / kbs;
        zs.push_back(splits);
        ztot += splits;
    }
    c->splitk.ensure((size_t)ztot * M * N * sizeof(float2));
    int z0 = 0, ci_ = 0;
    for (int kc0 = 0; kc0 < nkb; kc0 += kchunk, ++ci_) {
        const int nkbl = std::min(kchunk, nkb - kc0);
        const int splits = zs[ci_];
        const int kbs = (nkbl + splits - 1) / splits;
        const unsigned char* Af;
        long astride, akb0;
        if (table) {
            Af = c->beta32_gfmt.as<unsigned char>();
            astride = nkb;
            akb0 = kc0;
        } else {
            c->gfmt_a.ensure((size_t)itiles * nkbl * a_stage);
            rows(c->gfmt_a.as<unsigned char>(), kc0, nkbl);
            Af = c->gfmt_a.as<unsigned char>();
            astride = nkbl;
            akb0 = 0;
        }
        c->gfmt_b.ensure((size_t)jtiles * nkbl * b_stage);
        {
            const float2* Bk = B + (long)kc0 * 8;  // the chunk's first complex k
            const long thr = (long)jtiles * (TJ / 8) * nkbl * 32;
            fmt_rot_kernel<<<(int)std::min<long>(152 * 16, (thr + 255) / 256), 256, 0, c->stream>>>(
                Bk, ldb, bmap, N, K - kc0 * 8, TJ, jtiles, nkbl, c->gfmt_b.as<unsigned char>());
        }
        dim3 g(itiles, jtiles, splits);
        tcq_gram_kernel<<<g, QTHREADS, QSMEM, c->stream>>>(M, N, TJ, nkbl, kbs, Af, astride, akb0,
                                                           c->gfmt_b.as<unsigned char>(), c->splitk.as<float2>(), z0,
                                                           ctx_errflag(c));
        FS_CUDA(cudaGetLastError());
        z0 += splits;
    }
    long total = (long)M * N;
    int rb = (int)std::min<long>(2048, (total + 255) / 256);
    tc_gram_reduce_kernel<<<rb, 256, 0, c->stream>>>(M, N, ztot, c->splitk.as<float2>(), C, ci, cj, alpha, beta);
    FS_CUDA(cudaGetLastError());
}

template <typename A2>
void tc_gemm_nn(fs_ctx* c, int M, int N, int K, const A2* A, long ai, long ak, const float2* B, long ldb,
                const int* bmap, float2* C, long ldc, const int* cmap, double alpha, double beta, const float2* D,
                long ldd, int kid, const BetaGen* gen) {
    if (M <= 0 || N <= 0) return;
    set_attrs();
    ProfScope ps(c, kid, ((double)K + M * (beta != 0.0 ? 2.0 : 1.0)) * N * sizeof(float2) + (double)M * K * sizeof(A2),
                 8.0 * M * N * K);
    const int nkb = std::max(1, (K + 7) / 8);
    const int itiles = (M + TN_MAX - 1) / TN_MAX;
    const int TI = (((M + itiles - 1) / itiles) + 15) / 16 * 16;  // balanced tiles, a multiple of 16 columns
    const int gtiles = (N + 63) / 64;
    const size_t col_bytes = (size_t)nkb * 2 * QA_BYTES;         // A images of one plane-wave tile
    auto expand = [&](int gs, int ng, unsigned char* dst) {
        const long total = (long)ng * 64 * nkb * 4;
        const int nbk = (int)std::min<long>(152 * 16, (total + 255) / 256);
        if (gen)
            fmt_beta_expand_kernel<<<nbk, 256, 0, c->stream>>>(*gen, K, N, nkb, gs * 64, ng, dst);
        else
            fmt_expand_kernel<<<nbk, 256, 0, c->stream>>>(B, ldb, bmap, K, N, nkb, gs * 64, ng, dst);
    };
    bool table = !gen && B == c->beta32.as<float2>() && bmap == nullptr && N == c->npw && K == c->nptot;
    if (table && !c->beta32_fmt.p && (size_t)gtiles * col_bytes <= FS_TABLE_FMT_MAX_BYTES) {
        c->beta32_fmt.alloc((size_t)gtiles * col_bytes);
        expand(0, gtiles, c->beta32_fmt.as<unsigned char>());
    }
    table = table && c->beta32_fmt.p != nullptr;
    c->bfmt.ensure((size_t)itiles * nkb * 2 * (size_t)TI * QK * 4);
    {
        const long total = (long)itiles * TI * nkb * 4;
        fmt_coef_kernel<A2><<<(int)std::min<long>(152 * 16, (total + 255) / 256), 256, 0, c->stream>>>(
            A, ai, ak, M, K, TI, itiles, nkb, c->bfmt.as<unsigned char>());
    }
    const int chunk = table ? gtiles : (int)std::max<size_t>(1, std::min<size_t>(gtiles, FS_FMT_CHUNK_BYTES / col_bytes));
    // ring of the persistent kernel: as many stages of this tile size as fit
    const size_t sbytes = (size_t)2 * QA_BYTES + (size_t)2 * TI * QK * 4;
    const int nst = (int)std::min<size_t>(QS_MAX, (QSMEM_MAX - QCTL_BYTES) / sbytes);
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        FS_CUDA(cudaGetDevice(&dev));
        FS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    for (int gs = 0; gs < gtiles; gs += chunk) {
        const int ng = std::min(chunk, gtiles - gs);
        const unsigned char* Af;
        if (table) {
            Af = c->beta32_fmt.as<unsigned char>() + (size_t)gs * col_bytes;
        } else {
            c->afmt.ensure((size_t)ng * col_bytes);
            expand(gs, ng, c->afmt.as<unsigned char>());
            Af = c->afmt.as<unsigned char>();
        }
        const int ntiles = itiles * ng;
        const int grid = std::min(ntiles, nsm);
        tcq_nn_kernel<<<grid, QTHREADS, (size_t)nst * sbytes + QCTL_BYTES, c->stream>>>(
            M, N, nkb, TI, itiles, ntiles, gs, nst, Af, c->bfmt.as<unsigned char>(), C, ldc, cmap, (float)alpha,
            (float)beta, D, ldd, ctx_errflag(c));
        FS_CUDA(cudaGetLastError());
    }
}

template void tc_gemm_nn<double2>(fs_ctx*, int, int, int, const double2*, long, long, const float2*, long, const int*,
                                  float2*, long, const int*, double, double, const float2*, long, int, const BetaGen*);
template void tc_gemm_nn<float2>(fs_ctx*, int, int, int, const float2*, long, long, const float2*, long, const int*,
                                 float2*, long, const int*, double, double, const float2*, long, int, const BetaGen*);

extern "C" fs_status fs_wait_selftest(fs_ctx* c, long long polls) {
    if (!c) return FS_ERR_ARG;
    if (polls < 1 || polls > (1ll << 24)) {
        c->err = "fs_wait_selftest: polls out of range [1, 2^24]";
        return FS_ERR_ARG;
    }
    try {
        wait_selftest_kernel<<<1, 32, 0, c->stream>>>(polls, ctx_errflag(c));
        FS_CUDA(cudaGetLastError());
        ctx_check_errflag(c);
        c->err.clear();
        return FS_OK;
    } catch (const fs_error& e) {
        c->err = e.msg;
        return e.code;
    }
}
