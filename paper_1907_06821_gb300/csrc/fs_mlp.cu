// Learned G-shell preconditioner: a 4 -> 128 -> 128 -> 128 -> 1 perceptron
// that scales the paper's M(G) per band and per kinetic-energy shell,
//     W_G = M(G) exp(z_{i, s(G)}) R_G,   z = f(features of (band i, shell s)),
// with its forward pass, backward pass (weighted MSE on log-gain labels) and
// Adam update as kernels here.  Parameter layout (flat FP32, master copy):
//     W1[128][4] b1[128] W2[128][128] b2[128] W3[128][128] b3[128] W4[128] b4
// Training (forward and backward) reads the weights rounded to BF16 with FP32
// arithmetic on CUDA cores; inference runs the two 128 x 128 layers on the tensor
// cores with BF16 operands and FP32 accumulation; the master copy and the
// gradients stay FP32.
// Features: (shell centre / ecut, log10 shell share of |R|^2, d_i / 0.1 Ha,
// log10 ||R_i|| / 10).  The output layer starts at zero, so the untrained
// network is exactly the paper's M(G).
#include "fs_common.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <random>

namespace {

constexpr int H = 128;           // hidden width
constexpr int TR = 28;           // rows per block (3 x TR x 128 floats of shared memory)
constexpr int P_W1 = 0, P_B1 = P_W1 + H * 4, P_W2 = P_B1 + H, P_B2 = P_W2 + H * H, P_W3 = P_B2 + H,
              P_B3 = P_W3 + H * H, P_W4 = P_B3 + H, P_B4 = P_W4 + H, NPARAM = P_B4 + 1;

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Wt1[k][j] = bf(W1[j][k]) etc.: transposed BF16-rounded copies for coalesced reads
__global__ void mlp_prepare_kernel(const float* __restrict__ P, float* __restrict__ T) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < H * 4) {
        int k = t / H, j = t % H;
        T[P_W1 + t] = bf(P[P_W1 + j * 4 + k]);
    }
    if (t < H * H) {
        int k = t / H, j = t % H;
        T[P_W2 + t] = bf(P[P_W2 + j * H + k]);
        T[P_W3 + t] = bf(P[P_W3 + j * H + k]);
    }
    if (t < H) {
        T[P_B1 + t] = P[P_B1 + t];
        T[P_B2 + t] = P[P_B2 + t];
        T[P_B3 + t] = P[P_B3 + t];
        T[P_W4 + t] = bf(P[P_W4 + t]);
    }
    if (t == 0) T[P_B4] = P[P_B4];
}

// forward for a tile of TR rows; leaves h1, h2, h3 in shared memory and z in zsh
__device__ void mlp_tile_forward(const float* __restrict__ T, const float* __restrict__ F, int row0, int rows,
                                 float (*h1)[H], float (*h2)[H], float (*h3)[H], float* zsh, float* red) {
    const int j = threadIdx.x;
    for (int r = 0; r < TR; ++r) {
        int row = row0 + r;
        float a = T[P_B1 + j];
        if (row < rows) {
#pragma unroll
            for (int k = 0; k < 4; ++k) a += T[P_W1 + k * H + j] * F[(long)row * 4 + k];
        }
        h1[r][j] = tanhf(a);
    }
    __syncthreads();
    float acc[TR];
#pragma unroll
    for (int r = 0; r < TR; ++r) acc[r] = T[P_B2 + j];
    for (int k = 0; k < H; ++k) {
        float w = T[P_W2 + k * H + j];
#pragma unroll
        for (int r = 0; r < TR; ++r) acc[r] += w * h1[r][k];
    }
#pragma unroll
    for (int r = 0; r < TR; ++r) h2[r][j] = tanhf(acc[r]);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TR; ++r) acc[r] = T[P_B3 + j];
    for (int k = 0; k < H; ++k) {
        float w = T[P_W3 + k * H + j];
#pragma unroll
        for (int r = 0; r < TR; ++r) acc[r] += w * h2[r][k];
    }
#pragma unroll
    for (int r = 0; r < TR; ++r) h3[r][j] = tanhf(acc[r]);
    __syncthreads();
    // z[r] = b4 + sum_j W4[j] h3[r][j]: per-thread products, reduced per row
    const float w4 = T[P_W4 + j];
    for (int r = 0; r < TR; ++r) {
        float v = w4 * h3[r][j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((j & 31) == 0) red[r * 4 + (j >> 5)] = v;
    }
    __syncthreads();
    if (j < TR) zsh[j] = T[P_B4] + red[j * 4] + red[j * 4 + 1] + red[j * 4 + 2] + red[j * 4 + 3];
    __syncthreads();
}

// ------------------------------------------------------------------ tensor-core forward
// Inference on the 5th-generation tensor cores: tiles of 128 rows, one thread per
// row; layer 1 (K = 4) and layer 4 (N = 1) on CUDA cores, layers 2 and 3 as
// tcgen05.mma kind::f16 with BF16 operands (the BF16 weights and the hidden
// activations rounded to BF16) and FP32 accumulation in tensor memory (128 x 128).
// Operands sit in shared memory in the K-major core-matrix layout (8 rows x 16 bytes
// per core matrix, 16 core matrices along K); each MMA takes K = 16.
constexpr int MT = 128;                               // rows per tile (UMMA M)
constexpr int OP_BYTES = MT * H * 2;                  // one 128 x 128 BF16 operand (32 KB)
constexpr int TC_SMEM = 3 * OP_BYTES + 64;            // W2, W3, activations, barrier + slot
constexpr long long TC_WAIT_LIMIT = 1ll << 26;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) of a 128 x 128 BF16 K-major operand
__device__ __forceinline__ uint32_t kmaj_bf16(int row, int k) {
    return (uint32_t)((((row >> 3) * (H / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint64_t sdesc_bf16(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;               // leading byte offset: next core matrix along K
    d |= (uint64_t)(((H / 8) * 128) >> 4) << 32;   // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;
    return d;
}

// kind::f16, BF16 A and B, FP32 D, K-major both, M = N = 128
constexpr uint32_t IDESC_BF16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(H >> 3) << 17) |
                                ((uint32_t)(MT >> 4) << 24);

__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_addr(bar);
    for (long long it = 0; it < TC_WAIT_LIMIT; ++it) {
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

// the 8 MMAs of one layer: D = A W^T over K = 128, then a commit to bar
__device__ __forceinline__ void tc_layer_mma(uint32_t tmem, uint32_t a, uint32_t w, uint64_t* bar) {
#pragma unroll
    for (int ks = 0; ks < H / 16; ++ks) {
        const uint64_t ad = sdesc_bf16(a + ks * 256), bd = sdesc_bf16(w + ks * 256);
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(tmem), "l"(ad), "l"(bd), "r"(IDESC_BF16), "r"(ks > 0 ? 1u : 0u));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// 32 consecutive accumulator columns of this thread's row (lane quadrant of its warp)
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
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

// 8 BF16 values as one 16-byte chunk
__device__ __forceinline__ uint4 pack8(const float* v) {
    uint4 o;
    uint32_t* w = reinterpret_cast<uint32_t*>(&o);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(v[2 * i]));
        const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(v[2 * i + 1]));
        w[i] = lo | (hi << 16);
    }
    return o;
}

// the activation row of this thread: tanh(accumulator + bias) into the A operand
// (BF16), or, for the last hidden layer, dotted with W4 (FP32) into z
__device__ __forceinline__ float tc_drain(uint32_t tmem, const float* __restrict__ bias, unsigned char* act,
                                          const float* __restrict__ w4, int row) {
    const int warp = threadIdx.x >> 5;
    float zsum = 0.f;
#pragma unroll
    for (int c = 0; c < H / 32; ++c) {
        float v[32];
        tc_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * c), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = tanhf(v[i] + bias[32 * c + i]);
        if (act) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                *reinterpret_cast<uint4*>(act + kmaj_bf16(row, 32 * c + 8 * q)) = pack8(v + 8 * q);
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) zsum += w4[32 * c + i] * v[i];
        }
    }
    return zsum;
}

__global__ void __launch_bounds__(MT, 1) mlp_forward_tc_kernel(const float* __restrict__ P,
                                                              const float* __restrict__ T,
                                                              const float* __restrict__ F, int rows,
                                                              float* __restrict__ z, int* errflag) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* w2 = smem;
    unsigned char* w3 = smem + OP_BYTES;
    unsigned char* act = smem + 2 * OP_BYTES;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 3 * OP_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 3 * OP_BYTES + 8);
    __shared__ float w1s[H * 4], b1s[H], b2s[H], b3s[H], w4s[H];
    const int t = threadIdx.x;
    // weights: W2, W3 (row n = output, K = input) as BF16 operands; the rest as the
    // CUDA-core forward reads them (T: BF16-rounded W1 and W4, FP32 biases)
    for (int e = t; e < H * H; e += MT) {
        const int n = e / H, k = e % H;
        *reinterpret_cast<__nv_bfloat16*>(w2 + kmaj_bf16(n, k)) = __float2bfloat16_rn(P[P_W2 + e]);
        *reinterpret_cast<__nv_bfloat16*>(w3 + kmaj_bf16(n, k)) = __float2bfloat16_rn(P[P_W3 + e]);
    }
    for (int e = t; e < H * 4; e += MT) w1s[e] = T[P_W1 + e];
    b1s[t] = T[P_B1 + t];
    b2s[t] = T[P_B2 + t];
    b3s[t] = T[P_B3 + t];
    w4s[t] = T[P_W4 + t];
    const float b4 = T[P_B4];
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (t < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(H));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t a_s = smem_addr(act), w2_s = smem_addr(w2), w3_s = smem_addr(w3);
    uint32_t phase = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile * MT < rows && ok; tile += gridDim.x) {
        const int row = tile * MT + t;
        // layer 1 on CUDA cores, into the A operand (BF16)
        float f[4] = {0.f, 0.f, 0.f, 0.f};
        if (row < rows)
#pragma unroll
            for (int k = 0; k < 4; ++k) f[k] = F[(long)row * 4 + k];
#pragma unroll
        for (int c = 0; c < H / 8; ++c) {
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int j = 8 * c + i;
                float a = b1s[j];
#pragma unroll
                for (int k = 0; k < 4; ++k) a += w1s[k * H + j] * f[k];
                v[i] = tanhf(a);
            }
            *reinterpret_cast<uint4*>(act + kmaj_bf16(t, 8 * c)) = pack8(v);
        }
        float zr = 0.f;
#pragma unroll
        for (int layer = 0; layer < 2; ++layer) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (t == 0) tc_layer_mma(tmem, a_s, layer == 0 ? w2_s : w3_s, bar);
            // every thread polls; the vote keeps each warp together if one gives up
            if (!__all_sync(0xffffffffu, tc_wait(bar, phase))) ok = false;
            phase ^= 1;
            if (!__syncthreads_and(ok)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (layer == 0)
                tc_drain(tmem, b2s, act, nullptr, t);
            else
                zr = tc_drain(tmem, b3s, nullptr, w4s, t);
        }
        if (ok && row < rows) z[row] = b4 + zr;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (!ok && t == 0) atomicExch(errflag, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (t < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(H));
}

// Loss sum_r w_r (z_r - t_r)^2 * inv_sw and its gradient, one partial per block.
// The backward pass uses the FP32 master weights (dz/dh) with the BF16 forward
// activations.
__global__ void __launch_bounds__(H) mlp_backward_kernel(const float* __restrict__ P, const float* __restrict__ T,
                                                         const float* __restrict__ F, const float* __restrict__ zt,
                                                         const float* __restrict__ wt, int rows, float inv_sw,
                                                         float* __restrict__ gpart, float* __restrict__ lpart) {
    __shared__ float h1[TR][H], h2[TR][H], h3[TR][H];
    __shared__ float zsh[TR], red[TR * 4], g[TR];
    const int row0 = blockIdx.x * TR;
    const int j = threadIdx.x;
    mlp_tile_forward(T, F, row0, rows, h1, h2, h3, zsh, red);
    float* gp = gpart + (long)blockIdx.x * NPARAM;
    if (j < TR) {
        int row = row0 + j;
        float r = 0.f, w = 0.f;
        if (row < rows) {
            r = zsh[j] - zt[row];
            w = wt[row];
        }
        g[j] = 2.f * w * r * inv_sw;
        red[j] = w * r * r * inv_sw;
    }
    __syncthreads();
    if (j == 0) {
        float l = 0.f, gb = 0.f;
        for (int r = 0; r < TR; ++r) {
            l += red[r];
            gb += g[r];
        }
        lpart[blockIdx.x] = l;
        gp[P_B4] = gb;
    }
    // layer 4
    {
        float s = 0.f;
        for (int r = 0; r < TR; ++r) s += g[r] * h3[r][j];
        gp[P_W4 + j] = s;
    }
    // delta3 -> stored over h3 after use; need h3 for gW4 (done) and the tanh derivative
    const float w4 = P[P_W4 + j];
    __syncthreads();
    for (int r = 0; r < TR; ++r) h3[r][j] = g[r] * w4 * (1.f - h3[r][j] * h3[r][j]);  // delta3[r][j]
    __syncthreads();
    // layer 3: gW3[j][k] = sum_r delta3[r][j] h2[r][k]; gb3[j] = sum_r delta3[r][j]
    {
        float sb = 0.f;
        for (int r = 0; r < TR; ++r) sb += h3[r][j];
        gp[P_B3 + j] = sb;
        for (int k = 0; k < H; ++k) {
            float s = 0.f;
#pragma unroll 8
            for (int r = 0; r < TR; ++r) s += h3[r][j] * h2[r][k];
            gp[P_W3 + j * H + k] = s;
        }
    }
    // delta2[r][k] = (sum_j delta3[r][j] W3[j][k]) (1 - h2^2): thread = k
    float acc[TR];
#pragma unroll
    for (int r = 0; r < TR; ++r) acc[r] = 0.f;
    for (int jj = 0; jj < H; ++jj) {
        float w = P[P_W3 + jj * H + j];
#pragma unroll
        for (int r = 0; r < TR; ++r) acc[r] += h3[r][jj] * w;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TR; ++r) h2[r][j] = acc[r] * (1.f - h2[r][j] * h2[r][j]);  // delta2
    __syncthreads();
    {
        float sb = 0.f;
        for (int r = 0; r < TR; ++r) sb += h2[r][j];
        gp[P_B2 + j] = sb;
        for (int k = 0; k < H; ++k) {
            float s = 0.f;
#pragma unroll 8
            for (int r = 0; r < TR; ++r) s += h2[r][j] * h1[r][k];
            gp[P_W2 + j * H + k] = s;
        }
    }
#pragma unroll
    for (int r = 0; r < TR; ++r) acc[r] = 0.f;
    for (int jj = 0; jj < H; ++jj) {
        float w = P[P_W2 + jj * H + j];
#pragma unroll
        for (int r = 0; r < TR; ++r) acc[r] += h2[r][jj] * w;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TR; ++r) h1[r][j] = acc[r] * (1.f - h1[r][j] * h1[r][j]);  // delta1
    __syncthreads();
    {
        float sb = 0.f;
        float s4[4] = {0.f, 0.f, 0.f, 0.f};
        for (int r = 0; r < TR; ++r) {
            int row = row0 + r;
            float d = h1[r][j];
            sb += d;
            if (row < rows) {
#pragma unroll
                for (int k = 0; k < 4; ++k) s4[k] += d * F[(long)row * 4 + k];
            }
        }
        gp[P_B1 + j] = sb;
#pragma unroll
        for (int k = 0; k < 4; ++k) gp[P_W1 + j * 4 + k] = s4[k];
    }
}

// fixed-order sum over blocks (deterministic)
__global__ void sum_parts_kernel(const float* __restrict__ part, int nblk, int n, float* __restrict__ out) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double s = 0;
    for (int b = 0; b < nblk; ++b) s += part[(long)b * n + p];
    out[p] = (float)s;
}

__global__ void adam_kernel(float* P, const float* __restrict__ g, float* m, float* v, int n, float lr, float bc1,
                            float bc2) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float gg = g[p];
    float mm = 0.9f * m[p] + 0.1f * gg;
    float vv = 0.999f * v[p] + 0.001f * gg * gg;
    m[p] = mm;
    v[p] = vv;
    P[p] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + 1e-8f);
}

// per (band a, shell s): sum over the shell of |R|^2 (and, with E, of |E|^2
// and |M R|^2); shells are contiguous ranges of a permutation
template <typename T2>
__global__ void shell_stats_kernel(const T2* __restrict__ R, const int* __restrict__ act, const T2* __restrict__ Err,
                                   long npw, const int* __restrict__ perm, const int* __restrict__ off,
                                   const double* __restrict__ M, int nshell, double* __restrict__ r2,
                                   double* __restrict__ num, double* __restrict__ den) {
    __shared__ double sh[3][256];
    const int s = blockIdx.x, a = blockIdx.y;
    const long band = act ? act[a] : a;
    const T2* r = R + band * npw;
    const T2* e = Err ? Err + (long)a * npw : nullptr;
    double s0 = 0, s1 = 0, s2 = 0;
    for (int t = off[s] + threadIdx.x; t < off[s + 1]; t += blockDim.x) {
        int gidx = perm[t];
        T2 v = r[gidx];
        double p = (double)v.x * v.x + (double)v.y * v.y;
        s0 += p;
        if (e) {
            double mm = M[gidx];
            T2 q = e[gidx];
            s1 += (double)q.x * q.x + (double)q.y * q.y;
            s2 += mm * mm * p;
        }
    }
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    sh[2][threadIdx.x] = s2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        r2[(long)a * nshell + s] = sh[0][0];
        if (e) {
            num[(long)a * nshell + s] = sh[1][0];
            den[(long)a * nshell + s] = sh[2][0];
        }
    }
}

constexpr double LABEL_LO = -2.302585092994046;  // log 0.1
constexpr double LABEL_HI = 2.302585092994046;   // log 10

// features of (band a, shell s) from the shell sums; labels/weights when num != null
__global__ void features_kernel(const double* __restrict__ r2, const double* __restrict__ num,
                                const double* __restrict__ den, const double2* __restrict__ dots,
                                const int* __restrict__ act, const int* __restrict__ off, int na, int nshell,
                                long npw, float* __restrict__ F, float* __restrict__ zt, float* __restrict__ wt) {
    int a = blockIdx.x;
    if (a >= na) return;
    __shared__ double tot, dtot, ntot;
    if (threadIdx.x == 0) {
        double t = 0, dt = 0, nt = 0;
        for (int s = 0; s < nshell; ++s) {
            t += r2[(long)a * nshell + s];
            if (den) dt += den[(long)a * nshell + s];
            if (num) nt += num[(long)a * nshell + s];
        }
        tot = t;
        dtot = dt;
        ntot = nt;
    }
    __syncthreads();
    const int band = act ? act[a] : a;
    const double d = dots[band].x;
    const double mean_all = tot / (double)npw;
    for (int s = threadIdx.x; s < nshell; s += blockDim.x) {
        long row = (long)a * nshell + s;
        int cnt = off[s + 1] - off[s];
        double ms = cnt > 0 ? r2[row] / cnt : 0.0;
        F[row * 4 + 0] = (float)((s + 0.5) / nshell);
        F[row * 4 + 1] = (float)fmax(log10(fmax(ms, 1e-300) / fmax(mean_all, 1e-300)), -30.0);
        F[row * 4 + 2] = (float)(d / 0.1);
        F[row * 4 + 3] = (float)(log10(fmax(sqrt(tot), 1e-300)) / 10.0);
        if (num) {
            // log of the shell's share of the error over its share of the
            // preconditioned residual, halved (a ratio of magnitudes), clipped
            // to [log 0.1, log 10]; weight: the shell's share of |M R|^2
            const double b = dtot > 0 ? den[row] / dtot : 0.0;
            const double an = ntot > 0 ? num[row] / ntot : 0.0;
            double z = 0.0;
            if (b > 0) z = an > 0 ? 0.5 * log(an / b) : LABEL_LO;
            zt[row] = (float)fmin(fmax(z, LABEL_LO), LABEL_HI);
            wt[row] = (float)b;
        }
    }
}

// W[a] = M(q) exp(z[a][shell(q)]) R[act[a]]
// (M(G) evaluated exactly as the plain preconditioner kernel does, so that a
// zero network output reproduces it bit for bit)
template <typename T2>
__global__ void make_w_learned_kernel(const T2* __restrict__ R, const int* __restrict__ act, long npw,
                                      T2* __restrict__ W, const double* __restrict__ kin, double e_ref, double dE2,
                                      const int* __restrict__ shell_of, const float* __restrict__ z, int nshell) {
    using Rl = typename real_of<T2>::t;
    const int a = blockIdx.y;
    const long band = act[a];
    const T2* r = R + band * npw;
    T2* w = W + (long)a * npw;
    const float* za = z + (long)a * nshell;
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < npw; g += (long)gridDim.x * blockDim.x) {
        double d = kin[g] - e_ref;
        double m = 1.0 / (d * d + dE2);
        const float zz = za[shell_of[g]];
        if (zz != 0.f) m *= exp((double)zz);
        T2 v = r[g];
        w[g] = mk((Rl)m * v.x, (Rl)m * v.y);
    }
}

// E[a] = X_ref X_ref^H x_i - x_i, the correction that takes band i into the reference span
template <typename T2>
__global__ void err_from_proj_kernel(const T2* __restrict__ proj, const T2* __restrict__ X, const int* __restrict__ act,
                                     long npw, T2* __restrict__ E) {
    using Rl = typename real_of<T2>::t;
    const int a = blockIdx.y;
    const long band = act[a];
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < npw; g += (long)gridDim.x * blockDim.x) {
        T2 p = proj[(long)a * npw + g], x = X[band * npw + g];
        E[(long)a * npw + g] = mk((Rl)(p.x - x.x), (Rl)(p.y - x.y));
    }
}

}  // namespace

// ------------------------------------------------------------------ host side
int mlp_nparam() { return NPARAM; }

void mlp_setup(fs_ctx* c) {
    Mlp& L = c->mlp;
    if (L.ready) return;
    L.nshell = 32;
    const int ns = L.nshell;
    // shells: uniform bins of |q|^2/2 over [0, ecut]; permutation grouping each shell
    std::vector<int> shell(c->npw), cnt(ns + 1, 0), perm(c->npw);
    for (int g = 0; g < c->npw; ++g) {
        int s = (int)std::floor(c->kin_h[g] / c->ecut * ns);
        s = std::min(std::max(s, 0), ns - 1);
        shell[g] = s;
        cnt[s + 1]++;
    }
    for (int s = 0; s < ns; ++s) cnt[s + 1] += cnt[s];
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    for (int g = 0; g < c->npw; ++g) perm[pos[shell[g]]++] = g;
    std::vector<double> M(c->npw);
    L.shell_of.alloc(c->npw * sizeof(int));
    L.perm.alloc(c->npw * sizeof(int));
    L.off.alloc((ns + 1) * sizeof(int));
    FS_CUDA(cudaMemcpy(L.shell_of.p, shell.data(), c->npw * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(L.perm.p, perm.data(), c->npw * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(L.off.p, cnt.data(), (ns + 1) * sizeof(int), cudaMemcpyHostToDevice));
    L.P.alloc(NPARAM * sizeof(float));
    L.T.alloc(NPARAM * sizeof(float));
    L.m.alloc(NPARAM * sizeof(float));
    L.v.alloc(NPARAM * sizeof(float));
    L.g.alloc(NPARAM * sizeof(float));
    // default initialisation: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) hidden layers, zero output layer
    std::vector<float> p(NPARAM, 0.f);
    std::mt19937 gen(1234);
    auto fill = [&](int o, int n, int fan) {
        std::uniform_real_distribution<float> d(-1.f / std::sqrt((float)fan), 1.f / std::sqrt((float)fan));
        for (int i = 0; i < n; ++i) p[o + i] = d(gen);
    };
    fill(P_W1, H * 4, 4);
    fill(P_B1, H, 4);
    fill(P_W2, H * H, H);
    fill(P_B2, H, H);
    fill(P_W3, H * H, H);
    fill(P_B3, H, H);
    FS_CUDA(cudaMemcpy(L.P.p, p.data(), NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemset(L.m.p, 0, NPARAM * sizeof(float)));
    FS_CUDA(cudaMemset(L.v.p, 0, NPARAM * sizeof(float)));
    L.step = 0;
    L.ready = true;
    mlp_prepare(c);
}

void mlp_prepare(fs_ctx* c) {
    mlp_prepare_kernel<<<(H * H + 255) / 256, 256, 0, c->stream>>>(c->mlp.P.as<float>(), c->mlp.T.as<float>());
    FS_CUDA(cudaGetLastError());
}

void mlp_forward(fs_ctx* c, const float* F, int rows, float* z) {
    if (rows <= 0) return;
    ProfScope ps(c, KS_VECTOR, rows * 20.0, rows * 2.0 * (4 * H + 2 * H * H + H));
    static bool attr = false;
    if (!attr) {
        FS_CUDA(cudaFuncSetAttribute((const void*)mlp_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     TC_SMEM));
        attr = true;
    }
    int dev = 0, nsm = 0;
    FS_CUDA(cudaGetDevice(&dev));
    FS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::max(1, std::min((rows + MT - 1) / MT, nsm));
    mlp_forward_tc_kernel<<<grid, MT, TC_SMEM, c->stream>>>(c->mlp.P.as<float>(), c->mlp.T.as<float>(), F, rows, z,
                                                            ctx_errflag(c));
    FS_CUDA(cudaGetLastError());
}

// loss (returned) and gradient (into c->mlp.g) of the weighted MSE on rows
double mlp_loss_grad(fs_ctx* c, const float* F, const float* zt, const float* wt, int rows, double sw) {
    Mlp& L = c->mlp;
    int nblk = (rows + TR - 1) / TR;
    L.gpart.ensure((size_t)nblk * NPARAM * sizeof(float));
    L.lpart.ensure((size_t)nblk * sizeof(float) + sizeof(float));
    mlp_backward_kernel<<<nblk, H, 0, c->stream>>>(L.P.as<float>(), L.T.as<float>(), F, zt, wt, rows,
                                                   (float)(1.0 / sw), L.gpart.as<float>(), L.lpart.as<float>());
    sum_parts_kernel<<<(NPARAM + 255) / 256, 256, 0, c->stream>>>(L.gpart.as<float>(), nblk, NPARAM, L.g.as<float>());
    float* lsum = L.lpart.as<float>() + nblk;
    sum_parts_kernel<<<1, 32, 0, c->stream>>>(L.lpart.as<float>(), nblk, 1, lsum);
    float loss = 0;
    FS_CUDA(cudaMemcpyAsync(&loss, lsum, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return loss;
}

void mlp_adam(fs_ctx* c, float lr) {
    Mlp& L = c->mlp;
    L.step += 1;
    float bc1 = 1.f - std::pow(0.9f, (float)L.step), bc2 = 1.f - std::pow(0.999f, (float)L.step);
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, c->stream>>>(L.P.as<float>(), L.g.as<float>(), L.m.as<float>(),
                                                             L.v.as<float>(), NPARAM, lr, bc1, bc2);
    FS_CUDA(cudaGetLastError());
    mlp_prepare(c);
}

// features for the active bands of a residual block R (and labels when Err != null)
template <typename T2>
void mlp_features(fs_ctx* c, const T2* R, const int* act, int na, const double2* dots, const T2* Err, float* F,
                  float* zt, float* wt) {
    Mlp& L = c->mlp;
    const int ns = L.nshell;
    L.r2.ensure((size_t)na * ns * sizeof(double));
    L.num.ensure((size_t)na * ns * sizeof(double));
    L.den.ensure((size_t)na * ns * sizeof(double));
    if (!L.Mdev.p) {
        std::vector<double> M(c->npw);
        for (int g = 0; g < c->npw; ++g) {
            double d = c->kin_h[g] - L.e_ref;
            M[g] = 1.0 / (d * d + c->opt.dE * c->opt.dE);
        }
        L.Mdev.alloc(c->npw * sizeof(double));
        FS_CUDA(cudaMemcpy(L.Mdev.p, M.data(), c->npw * sizeof(double), cudaMemcpyHostToDevice));
    }
    dim3 g(ns, na);
    shell_stats_kernel<T2><<<g, 256, 0, c->stream>>>(R, act, Err, c->npw, L.perm.as<int>(), L.off.as<int>(),
                                                     L.Mdev.as<double>(), ns, L.r2.as<double>(), L.num.as<double>(),
                                                     L.den.as<double>());
    features_kernel<<<na, 64, 0, c->stream>>>(L.r2.as<double>(), Err ? L.num.as<double>() : nullptr,
                                              Err ? L.den.as<double>() : nullptr, dots, act, L.off.as<int>(), na, ns,
                                              c->npw, F, zt, wt);
    FS_CUDA(cudaGetLastError());
}

template <typename T2>
void mlp_make_w(fs_ctx* c, const T2* R, const int* act, int na, T2* W, const double2* dots) {
    Mlp& L = c->mlp;
    const int rows = na * L.nshell;
    L.F.ensure((size_t)rows * 4 * sizeof(float));
    L.z.ensure((size_t)rows * sizeof(float));
    mlp_features<T2>(c, R, act, na, dots, nullptr, L.F.as<float>(), nullptr, nullptr);
    mlp_forward(c, L.F.as<float>(), rows, L.z.as<float>());
    dim3 g((unsigned)std::min<long>(64, (c->npw + 255) / 256), na);
    make_w_learned_kernel<T2><<<g, 256, 0, c->stream>>>(R, act, c->npw, W, c->kin.as<double>(), L.e_ref,
                                                         c->opt.dE * c->opt.dE, L.shell_of.as<int>(), L.z.as<float>(),
                                                         L.nshell);
    FS_CUDA(cudaGetLastError());
}

template <typename T2>
void mlp_err_from_proj(fs_ctx* c, const T2* proj, const T2* X, const int* act, int na, T2* E) {
    dim3 g((unsigned)std::min<long>(64, (c->npw + 255) / 256), na);
    err_from_proj_kernel<T2><<<g, 256, 0, c->stream>>>(proj, X, act, c->npw, E);
    FS_CUDA(cudaGetLastError());
}

template void mlp_features<float2>(fs_ctx*, const float2*, const int*, int, const double2*, const float2*, float*,
                                   float*, float*);
template void mlp_features<double2>(fs_ctx*, const double2*, const int*, int, const double2*, const double2*, float*,
                                    float*, float*);
template void mlp_make_w<float2>(fs_ctx*, const float2*, const int*, int, float2*, const double2*);
template void mlp_make_w<double2>(fs_ctx*, const double2*, const int*, int, double2*, const double2*);
template void mlp_err_from_proj<float2>(fs_ctx*, const float2*, const float2*, const int*, int, float2*);
template void mlp_err_from_proj<double2>(fs_ctx*, const double2*, const double2*, const int*, int, double2*);
