// Warm-start network: a multilayer perceptron whose products run on the
// 5th-generation tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// tensor memory), trained with Adam on FP32 master weights.
//
// GEMM convention: C[M x N] = A[M x K] . B[N x K]^T with A and B bfloat16,
// row-major (K contiguous), K a multiple of 16 (buffers are zero-padded along
// K); rows of A beyond M and of B beyond N read as zero. One CTA computes a
// 128-row block with all N <= 256 columns in one accumulator.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "lbif.h"

namespace {

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------------------
// PTX wrappers (tcgen05 / mbarrier)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// D[tmem] (+)= A[smem] . B[smem]^T, kind::f16 (BF16 in, FP32 accumulate)
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
        "%13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, no swizzle, K-major: the operand is laid
// out as 8-row x 16-byte core matrices; lbo = byte step between core
// matrices along K, sbo = byte step between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version; base offset 0; layout type 0 = no swizzle
    return d;
}

// instruction descriptor, kind::f16: D F32, A and B BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// ---------------------------------------------------------------------------
// GEMM with fused epilogue
// ---------------------------------------------------------------------------
enum { EPI_NONE = 0, EPI_GELU = 1, EPI_GELU_GRAD = 2 };

struct Gemm {
    const bf16* A;
    int lda;
    const bf16* B;
    int ldb;
    int M, N, K;
    const float* bias;  // per column, may be null
    int epi;
    const float* zprev; // EPI_GELU_GRAD: pre-activation multiplied in (ld = ldz)
    float* Z;           // FP32 result (after bias / gradient factor), may be null
    int ldz;
    bf16* H;            // bf16 of the activated result, row-major, may be null
    int ldh;
    bf16* HT;           // bf16 transposed, may be null
    int ldht;
    int* err;
};

constexpr int GEMM_KC = 64;  // K staged per round
constexpr long long WAIT_LIMIT = 1LL << 22;  // try_wait polls; seconds at most

// shared memory of one CTA: two stages of A (128 x 64) and B (ntile x 64)
// bf16 tiles, then two mbarriers and the TMEM address slot
__host__ __device__ inline int gemm_stage_bytes(int ntile) { return (128 + ntile) * GEMM_KC * 2; }
__host__ __device__ inline int gemm_smem_bytes(int ntile) { return 2 * gemm_stage_bytes(ntile) + 32; }
__host__ __device__ inline uint32_t tmem_cols(int ntile)
{
    uint32_t c = 32;
    while (c < (uint32_t)ntile) c <<= 1;
    return c;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Issue the copies of K round k0 into a stage: A rows m0.., B rows n0.., as
// 8-row x 16-byte core matrices (K-major, no swizzle); rows past M / N read zero.
__device__ __forceinline__ void gemm_stage(const Gemm& g, uint8_t* sA, uint8_t* sB, int m0, int n0, int NT, int k0)
{
    const int kc = min(GEMM_KC, g.K - k0);  // multiple of 16
    const int kcore = kc / 8;
    for (int t = threadIdx.x; t < 128 * kcore; t += blockDim.x) {
        const int r = t / kcore, kp = t - r * kcore;
        const bool ok = m0 + r < g.M;
        const bf16* src = g.A + (size_t)(ok ? m0 + r : 0) * g.lda + k0 + kp * 8;
        cp_async16(sA + ((r >> 3) * kcore + kp) * 128 + (r & 7) * 16, src, ok);
    }
    for (int t = threadIdx.x; t < NT * kcore; t += blockDim.x) {
        const int r = t / kcore, kp = t - r * kcore;
        const bool ok = n0 + r < g.N;
        const bf16* src = g.B + (size_t)(ok ? n0 + r : 0) * g.ldb + k0 + kp * 8;
        cp_async16(sB + ((r >> 3) * kcore + kp) * 128 + (r & 7) * 16, src, ok);
    }
    cp_async_commit();
}

// Bounded wait of every thread on an mbarrier phase; one verdict per CTA.
__device__ __forceinline__ bool cta_wait(uint64_t* mbar, uint32_t parity)
{
    long long spins = 0;
    bool ok;
    while (!(ok = mbar_try_wait(mbar, parity)) && ++spins < WAIT_LIMIT) {
    }
    return __syncthreads_and(ok) != 0;
}

// One CTA: a 128-row block (blockIdx.x) x an ntile-column block (blockIdx.y)
// of C, accumulated in TMEM over K in rounds of 64; the copies of round k+1
// are in flight while the tensor core works on round k. GEMM_THREADS threads:
// the epilogue (bias, GELU, the FP32 and BF16 copies) dominates at K <= 256,
// and TMEM (ntile columns per CTA) caps the CTAs per SM, so the CTA is wide:
// warp w reads TMEM lanes 32 (w % 4) .. + 31 and every (GEMM_THREADS / 128)-th
// 16-column chunk, starting at chunk w / 4.
#ifndef LBIF_GEMM_THREADS
#define LBIF_GEMM_THREADS 256
#endif
constexpr int GEMM_THREADS = LBIF_GEMM_THREADS;
__global__ void __launch_bounds__(GEMM_THREADS, 2) k_gemm_tc(Gemm g, int ntile)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int SB = gemm_stage_bytes(ntile);
    uint64_t* mbar = (uint64_t*)(smem + 2 * SB);
    uint32_t* tslot = (uint32_t*)(mbar + 2);
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * ntile;
    const int NT = min(ntile, (g.N - n0 + 15) / 16 * 16);
    const uint32_t cols = tmem_cols(ntile);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (warp == 0) {
        tmem_alloc(tslot, cols);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        mbar_init(mbar, 1);
        mbar_init(mbar + 1, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = idesc_bf16(128, NT);
    uint32_t parity[2] = {0u, 0u};
    bool ok = true;
    const int nk = (g.K + GEMM_KC - 1) / GEMM_KC;

    gemm_stage(g, smem, smem + 128 * GEMM_KC * 2, m0, n0, NT, 0);
    for (int k = 0; k < nk && ok; ++k) {
        const int st = k & 1;
        uint8_t* sA = smem + st * SB;
        uint8_t* sB = sA + 128 * GEMM_KC * 2;
        if (k + 1 < nk) {
            // the other stage was read by the products of round k - 1
            if (k >= 1) {
                ok = cta_wait(mbar + (st ^ 1), parity[st ^ 1]);
                parity[st ^ 1] ^= 1u;
                if (!ok) break;
            }
            uint8_t* oA = smem + (st ^ 1) * SB;
            gemm_stage(g, oA, oA + 128 * GEMM_KC * 2, m0, n0, NT, (k + 1) * GEMM_KC);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        fence_proxy_async();  // copies of round k -> visible to the tensor core
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (threadIdx.x == 0) {
            const int kc = min(GEMM_KC, g.K - k * GEMM_KC);
            const uint32_t sbo = (kc / 8) * 128;
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
            for (int kk = 0; kk < kc / 16; ++kk)
                mma_bf16(tmem, smem_desc(a0 + kk * 256, 128, sbo), smem_desc(b0 + kk * 256, 128, sbo), idesc,
                         (k > 0 || kk > 0) ? 1u : 0u);
            mma_commit(mbar + st);
        }
    }
    // the last round's products (and, with one round only, the only ones)
    if (ok) {
        const int st = (nk - 1) & 1;
        ok = cta_wait(mbar + st, parity[st]);
        tc_fence_after();
    }

    if (ok) {
        // each thread owns one row (its TMEM lane) and 16 consecutive columns
        // per chunk: a full chunk is written with 16-byte vector stores
        const int lg = warp % 4, cg = warp / 4, ncg = GEMM_THREADS / 128;
        const int row = m0 + 32 * lg + lane;
        for (int c = 16 * cg; c < NT; c += 16 * ncg) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)c, v);
            if (row >= g.M) continue;
            const int nb = n0 + c;
            const bool full = nb + 16 <= g.N && (g.ldz % 4) == 0 && (g.ldh % 8) == 0;
            float z[16], h[16];
            float zp[16];
            if (g.epi == EPI_GELU_GRAD) {
                if (full) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 t = *reinterpret_cast<const float4*>(g.zprev + (size_t)row * g.ldz + nb + 4 * q);
                        zp[4 * q] = t.x, zp[4 * q + 1] = t.y, zp[4 * q + 2] = t.z, zp[4 * q + 3] = t.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) zp[j] = nb + j < g.N ? g.zprev[(size_t)row * g.ldz + nb + j] : 0.f;
                }
            }
            // the chunk's 16 biases: four 16-byte loads when aligned
            float bz[16];
            if (g.bias && nb + 16 <= g.N && ((uintptr_t)(g.bias + nb) & 15) == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 t = __ldg(reinterpret_cast<const float4*>(g.bias + nb) + q);
                    bz[4 * q] = t.x, bz[4 * q + 1] = t.y, bz[4 * q + 2] = t.z, bz[4 * q + 3] = t.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) bz[j] = (g.bias && nb + j < g.N) ? g.bias[nb + j] : 0.f;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                float zz = v[j] + bz[j];
                float hh = zz;
                if (g.epi == EPI_GELU) {
                    hh = gelu(zz);
                } else if (g.epi == EPI_GELU_GRAD) {
                    zz = zz * gelu_grad(zp[j]);
                    hh = zz;
                }
                z[j] = zz;
                h[j] = hh;
            }
            if (full) {
                if (g.Z) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<float4*>(g.Z + (size_t)row * g.ldz + nb + 4 * q) =
                            make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
                }
                if (g.H) {
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        uint4 pk;
                        uint32_t* w = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const __nv_bfloat162 b2 = __floats2bfloat162_rn(h[8 * q + 2 * e], h[8 * q + 2 * e + 1]);
                            w[e] = *reinterpret_cast<const uint32_t*>(&b2);
                        }
                        *reinterpret_cast<uint4*>(g.H + (size_t)row * g.ldh + nb + 8 * q) = pk;
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (nb + j >= g.N) break;
                    if (g.Z) g.Z[(size_t)row * g.ldz + nb + j] = z[j];
                    if (g.H) g.H[(size_t)row * g.ldh + nb + j] = __float2bfloat16_rn(h[j]);
                }
            }
            if (g.HT) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (nb + j >= g.N) break;
                    g.HT[(size_t)(nb + j) * g.ldht + row] = __float2bfloat16_rn(h[j]);
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(g.err, 1);
    }
    cp_async_wait<0>();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, cols);
}

// ---------------------------------------------------------------------------
// element-wise kernels
// ---------------------------------------------------------------------------
// X (batch x nin, FP32) -> bf16 rows (bp x kpad) and transposed (kpad x bp), zero padded
__global__ void k_pack_input(const float* X, int batch, int nin, int bp, int kpad, bf16* H, bf16* HT)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= bp * kpad) return;
    int r = i / kpad, c = i - r * kpad;
    float v = (r < batch && c < nin) ? X[(size_t)r * nin + c] : 0.f;
    bf16 b = __float2bfloat16_rn(v);
    H[i] = b;
    HT[(size_t)c * bp + r] = b;
}

// sum of the mask (one block, fixed order), at least 1
__global__ void k_msum(const float* mask, long long n, double* out)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += mask[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = fmax(sh[0], 1.0);
}

// dY = 2 mask (Y - T) / sum(mask): FP32 (bp x nout), bf16 rows (bp x opad) and
// bf16 transposed (nout x bp); per-block FP64 partial sums of the loss
__global__ void k_loss(const float* Y, const float* T, const float* mask, int batch, int nout, int opad, int bp,
                       const double* msum, float* dY, bf16* dYb, bf16* dYT, double* partial)
{
    __shared__ double sh[256];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < bp * nout) {
        int r = i / nout, c = i - r * nout;
        float d = 0.f;
        if (r < batch) {
            float m = mask[(size_t)r * nout + c];
            float e = (Y[(size_t)r * nout + c] - T[(size_t)r * nout + c]) * m;
            l = (double)e * e;
            d = (float)(2.0 * e / *msum);
        }
        dY[i] = d;
        bf16 b = __float2bfloat16_rn(d);
        dYb[(size_t)r * opad + c] = b;
        dYT[(size_t)c * bp + r] = b;
    }
    sh[threadIdx.x] = l;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// column sums of D (rows x cols, FP32) -> out (fixed-order, one thread per column)
__global__ void k_colsum(const float* D, int rows, int cols, float* out)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s += D[(size_t)r * cols + c];
    out[c] = (float)s;
}

// copy the first ncopy columns of a (rows x ld) FP32 matrix into dst (rows x ncopy)
__global__ void k_copy_cols(const float* src, int rows, int ld, int ncopy, float* dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * ncopy) return;
    int r = i / ncopy, c = i - r * ncopy;
    dst[i] = src[(size_t)r * ld + c];
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// bf16 shadows of W (nout x nin): row-major padded to kpad columns, and
// transposed (nin x opad, columns beyond nout stay zero)
__global__ void k_shadow(const float* W, int nout, int nin, int kpad, int opad, bf16* Wb, bf16* WTb)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nout * kpad) return;
    int r = i / kpad, c = i - r * kpad;
    float w = c < nin ? W[(size_t)r * nin + c] : 0.f;
    bf16 b = __float2bfloat16_rn(w);
    Wb[i] = b;
    if (c < nin) WTb[(size_t)c * opad + r] = b;
}

inline int up16(int v) { return (v + 15) / 16 * 16; }

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct lbif_mlp_ctx {
    int nin, hidden, nhidden, nout, max_batch, bp_max;
    int L;                      // layers
    std::vector<int> din, dout, kpad, opad;  // kpad, opad: widths rounded up to 16
    std::vector<long long> woff, boff;  // offsets into the flat parameter vector
    long long nparams;
    cudaStream_t stream = nullptr;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // flat FP32
    std::vector<bf16*> Wb, WTb;
    std::vector<float*> Z;       // pre-activations per layer (bp x dout)
    std::vector<bf16*> H, HT;    // layer inputs (bp x kpad) and transposed (kpad x bp)
    float* dY = nullptr;         // output error FP32 (bp x nout)
    std::vector<float*> dZ;      // per layer FP32 error (bp x dout)
    std::vector<bf16*> dZb, dZT; // bf16 copies
    float* dWtmp = nullptr;      // dW with padded columns
    float* Xd = nullptr;         // device staging for host inputs (max_batch x nin)
    float *Td = nullptr, *Md = nullptr, *Yd = nullptr;
    double* partial = nullptr;
    double* msum = nullptr;
    int* err = nullptr;
    long long adam_t = 0;
    std::string msg;
};

static thread_local std::string g_mlp_err = "no error";

static int mfail(lbif_mlp_ctx* m, int code, const std::string& s)
{
    if (m) m->msg = s;
    g_mlp_err = s;
    return code;
}

#define MCK(m, call)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return mfail((m), LBIF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static void mlp_free(lbif_mlp_ctx* m)
{
    if (!m) return;
    std::vector<void*> bufs = {m->p, m->g, m->m, m->v, m->dY, m->dWtmp, m->Xd, m->Td, m->Md, m->Yd, m->partial, m->msum, m->err};
    for (auto* b : m->Wb) bufs.push_back(b);
    for (auto* b : m->WTb) bufs.push_back(b);
    for (auto* b : m->Z) bufs.push_back(b);
    for (auto* b : m->H) bufs.push_back(b);
    for (auto* b : m->HT) bufs.push_back(b);
    for (auto* b : m->dZ) bufs.push_back(b);
    for (auto* b : m->dZb) bufs.push_back(b);
    for (auto* b : m->dZT) bufs.push_back(b);
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete m;
}

template <class T>
static bool dalloc(T** p, size_t n)
{
    if (cudaMalloc((void**)p, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return cudaMemset(*p, 0, sizeof(T) * (n ? n : 1)) == cudaSuccess;
}

extern "C" int lbif_mlp_create(lbif_mlp* out, int32_t nin, int32_t hidden, int32_t nhidden, int32_t nout,
                               int32_t max_batch, void* stream)
{
    if (!out || nin < 1 || nin > 256 || hidden < 16 || hidden > 256 || hidden % 16 || nhidden < 1 ||
        nout < 1 || nout > 256 || max_batch < 1)
        return mfail(nullptr, LBIF_ERR_ARG, "lbif_mlp_create: widths must be in [1, 256] (hidden a multiple of 16)");
    *out = nullptr;
    lbif_mlp_ctx* m = new lbif_mlp_ctx();
    m->nin = nin;
    m->hidden = hidden;
    m->nhidden = nhidden;
    m->nout = nout;
    m->max_batch = max_batch;
    m->bp_max = up16(max_batch);
    m->L = nhidden + 1;
    m->stream = (cudaStream_t)stream;
    long long off = 0;
    for (int l = 0; l < m->L; ++l) {
        int di = l == 0 ? nin : hidden, dq = l == m->L - 1 ? nout : hidden;
        m->din.push_back(di);
        m->dout.push_back(dq);
        m->kpad.push_back(up16(di));
        m->opad.push_back(up16(dq));
        m->woff.push_back(off);
        off += (long long)di * dq;
        m->boff.push_back(off);
        off += dq;
    }
    m->nparams = off;
    const int bp = m->bp_max;
    bool ok = dalloc(&m->p, off) && dalloc(&m->g, off) && dalloc(&m->m, off) && dalloc(&m->v, off) &&
              dalloc(&m->dY, (size_t)bp * nout) && dalloc(&m->dWtmp, (size_t)256 * 256) &&
              dalloc(&m->Xd, (size_t)max_batch * nin) && dalloc(&m->Td, (size_t)max_batch * nout) &&
              dalloc(&m->Md, (size_t)max_batch * nout) && dalloc(&m->Yd, (size_t)bp * nout) &&
              dalloc(&m->partial, (size_t)(bp * nout + 255) / 256 + 1) && dalloc(&m->msum, 1) &&
              dalloc(&m->err, 1);
    for (int l = 0; ok && l < m->L; ++l) {
        bf16 *wb, *wtb, *h, *ht, *dzb, *dzt;
        float *z, *dz;
        ok = dalloc(&wb, (size_t)m->dout[l] * m->kpad[l]) && dalloc(&wtb, (size_t)m->din[l] * m->opad[l]) &&
             dalloc(&z, (size_t)bp * m->dout[l]) && dalloc(&h, (size_t)bp * m->kpad[l]) &&
             dalloc(&ht, (size_t)m->kpad[l] * bp) && dalloc(&dz, (size_t)bp * m->dout[l]) &&
             dalloc(&dzb, (size_t)bp * m->opad[l]) && dalloc(&dzt, (size_t)m->dout[l] * bp);
        m->Wb.push_back(ok ? wb : nullptr);
        m->WTb.push_back(ok ? wtb : nullptr);
        m->Z.push_back(ok ? z : nullptr);
        m->H.push_back(ok ? h : nullptr);
        m->HT.push_back(ok ? ht : nullptr);
        m->dZ.push_back(ok ? dz : nullptr);
        m->dZb.push_back(ok ? dzb : nullptr);
        m->dZT.push_back(ok ? dzt : nullptr);
    }
    if (!ok) {
        mlp_free(m);
        return mfail(nullptr, LBIF_ERR_NOMEM, "lbif_mlp_create: device allocation failed");
    }
    if (cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, gemm_smem_bytes(256)) != cudaSuccess) {
        cudaGetLastError();
        mlp_free(m);
        return mfail(nullptr, LBIF_ERR_CUDA, "lbif_mlp_create: shared memory configuration failed");
    }
    *out = m;
    return LBIF_OK;
}

extern "C" int lbif_mlp_destroy(lbif_mlp m)
{
    if (!m) return mfail(nullptr, LBIF_ERR_ARG, "lbif_mlp_destroy: NULL handle");
    cudaStreamSynchronize(m->stream);
    mlp_free(m);
    return LBIF_OK;
}

extern "C" int64_t lbif_mlp_num_params(lbif_mlp m) { return m ? m->nparams : -1; }

extern "C" const char* lbif_mlp_last_error(lbif_mlp m) { return m ? m->msg.c_str() : g_mlp_err.c_str(); }

static int refresh_shadows(lbif_mlp_ctx* m)
{
    for (int l = 0; l < m->L; ++l) {
        int n = m->dout[l] * m->kpad[l];
        k_shadow<<<(n + 255) / 256, 256, 0, m->stream>>>(m->p + m->woff[l], m->dout[l], m->din[l], m->kpad[l],
                                                         m->opad[l], m->Wb[l], m->WTb[l]);
    }
    MCK(m, cudaGetLastError());
    return LBIF_OK;
}

extern "C" int lbif_mlp_set_params(lbif_mlp m, const float* params)
{
    if (!m || !params) return mfail(m, LBIF_ERR_ARG, "lbif_mlp_set_params: bad arguments");
    MCK(m, cudaMemcpyAsync(m->p, params, sizeof(float) * m->nparams, cudaMemcpyHostToDevice, m->stream));
    MCK(m, cudaMemsetAsync(m->m, 0, sizeof(float) * m->nparams, m->stream));
    MCK(m, cudaMemsetAsync(m->v, 0, sizeof(float) * m->nparams, m->stream));
    m->adam_t = 0;
    int rc = refresh_shadows(m);
    if (rc) return rc;
    MCK(m, cudaStreamSynchronize(m->stream));
    return LBIF_OK;
}

extern "C" int lbif_mlp_get_params(lbif_mlp m, float* params)
{
    if (!m || !params) return mfail(m, LBIF_ERR_ARG, "lbif_mlp_get_params: bad arguments");
    MCK(m, cudaMemcpyAsync(params, m->p, sizeof(float) * m->nparams, cudaMemcpyDeviceToHost, m->stream));
    MCK(m, cudaStreamSynchronize(m->stream));
    return LBIF_OK;
}

// Column block of a product: the whole N (<= 256) when there are enough row
// blocks to fill the GPU, else blocks of 64 columns for more CTAs.
static int gemm(lbif_mlp_ctx* m, const Gemm& g)
{
    if (g.N > 256 || g.K % 16 || g.K < 16)
        return mfail(m, LBIF_ERR_UNSUPPORTED, "gemm: N > 256 or K not a positive multiple of 16");
    const int mt = (g.M + 127) / 128;
    const int nfull = (g.N + 15) / 16 * 16;
    const int ntile = (mt >= 64 || nfull <= 64) ? nfull : 64;
    dim3 grid(mt, (g.N + ntile - 1) / ntile);
    // shared memory per CTA bounds the CTAs per SM so that their TMEM
    // columns (32..256 each) always fit in the SM's 512 together
    int smem = gemm_smem_bytes(ntile);
    if (tmem_cols(ntile) == 256 && smem < 80 * 1024) smem = 80 * 1024;
    k_gemm_tc<<<grid, GEMM_THREADS, smem, m->stream>>>(g, ntile);
    MCK(m, cudaGetLastError());
    return LBIF_OK;
}

static Gemm blank(lbif_mlp_ctx* m)
{
    Gemm g;
    memset(&g, 0, sizeof(g));
    g.err = m->err;
    return g;
}

// forward of `batch` rows already packed in H[0] / HT[0]. train: keep what
// back-propagation reads (every layer's FP32 pre-activation Z and the
// transposed BF16 activations HT); otherwise each hidden layer writes only
// the next layer's BF16 input, and the output goes to Yout (batch x nout,
// device memory) when given, else to Z of the last layer.
static int forward(lbif_mlp_ctx* m, int batch, bool train, float* Yout = nullptr)
{
    const int bp = up16(batch);
    for (int l = 0; l < m->L; ++l) {
        const bool last = l == m->L - 1;
        Gemm g = blank(m);
        g.A = m->H[l];
        g.lda = m->kpad[l];
        g.B = m->Wb[l];
        g.ldb = m->kpad[l];
        g.M = bp;
        g.N = m->dout[l];
        g.K = m->kpad[l];
        g.bias = m->p + m->boff[l];
        g.epi = last ? EPI_NONE : EPI_GELU;
        if (train || last) {
            g.Z = m->Z[l];
            g.ldz = m->dout[l];
        }
        if (last && !train && Yout) {
            g.Z = Yout;
            g.M = batch;  // the rows Yout holds
        }
        if (!last) {
            g.H = m->H[l + 1];
            g.ldh = m->kpad[l + 1];
            if (train) {
                g.HT = m->HT[l + 1];
                g.ldht = bp;
            }
        }
        int rc = gemm(m, g);
        if (rc) return rc;
    }
    return LBIF_OK;
}

static int pack_input(lbif_mlp_ctx* m, const float* X, int batch, int on_device)
{
    const float* Xd = X;
    if (!on_device) {
        MCK(m, cudaMemcpyAsync(m->Xd, X, sizeof(float) * (size_t)batch * m->nin, cudaMemcpyHostToDevice, m->stream));
        Xd = m->Xd;
    }
    const int bp = up16(batch);
    int n = bp * m->kpad[0];
    k_pack_input<<<(n + 255) / 256, 256, 0, m->stream>>>(Xd, batch, m->nin, bp, m->kpad[0], m->H[0], m->HT[0]);
    MCK(m, cudaGetLastError());
    return LBIF_OK;
}

static int check_err(lbif_mlp_ctx* m)
{
    int e = 0;
    MCK(m, cudaMemcpyAsync(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    MCK(m, cudaStreamSynchronize(m->stream));
    if (e) return mfail(m, LBIF_ERR_TIMEOUT, "tensor-core product did not complete within its wait limit");
    return LBIF_OK;
}

extern "C" int lbif_mlp_forward(lbif_mlp m, const float* X, int32_t batch, float* Y, int32_t on_device)
{
    if (!m || !X || !Y || batch < 1 || batch > m->max_batch)
        return mfail(m, LBIF_ERR_ARG, "lbif_mlp_forward: bad arguments");
    int rc = pack_input(m, X, batch, on_device);
    if (rc) return rc;
    // device output: the last product writes Y itself
    if ((rc = forward(m, batch, false, on_device ? Y : nullptr))) return rc;
    if (!on_device)
        MCK(m, cudaMemcpyAsync(Y, m->Z[m->L - 1], sizeof(float) * (size_t)batch * m->nout, cudaMemcpyDeviceToHost,
                               m->stream));
    return check_err(m);
}

// loss and gradients into m->g
static int backward(lbif_mlp_ctx* m, const float* T, const float* mask, int batch, int on_device, double* loss)
{
    const int bp = up16(batch);
    const int nout = m->nout;
    const float *Td = T, *Md = mask;
    if (!on_device) {
        MCK(m, cudaMemcpyAsync(m->Td, T, sizeof(float) * (size_t)batch * nout, cudaMemcpyHostToDevice, m->stream));
        MCK(m, cudaMemcpyAsync(m->Md, mask, sizeof(float) * (size_t)batch * nout, cudaMemcpyHostToDevice, m->stream));
        Td = m->Td;
        Md = m->Md;
    }
    const int L = m->L;
    const int n = bp * nout;
    const int nb = (n + 255) / 256;
    k_msum<<<1, 256, 0, m->stream>>>(Md, (long long)batch * nout, m->msum);
    k_loss<<<nb, 256, 0, m->stream>>>(m->Z[L - 1], Td, Md, batch, nout, m->opad[L - 1], bp, m->msum,
                                      m->dZ[L - 1], m->dZb[L - 1], m->dZT[L - 1], m->partial);
    MCK(m, cudaGetLastError());
    for (int l = L - 1; l >= 0; --l) {
        // dW_l = dZ_l^T . H_l  (M = dout, N = kpad_l, K = bp)
        Gemm gw = blank(m);
        gw.A = m->dZT[l];
        gw.lda = bp;
        gw.B = m->HT[l];
        gw.ldb = bp;
        gw.M = m->dout[l];
        gw.N = m->kpad[l];
        gw.K = bp;
        gw.Z = m->dWtmp;
        gw.ldz = m->kpad[l];
        int rc = gemm(m, gw);
        if (rc) return rc;
        int cnt = m->dout[l] * m->din[l];
        k_copy_cols<<<(cnt + 255) / 256, 256, 0, m->stream>>>(m->dWtmp, m->dout[l], m->kpad[l], m->din[l],
                                                              m->g + m->woff[l]);
        k_colsum<<<(m->dout[l] + 127) / 128, 128, 0, m->stream>>>(m->dZ[l], bp, m->dout[l], m->g + m->boff[l]);
        MCK(m, cudaGetLastError());
        if (l == 0) break;
        // dZ_{l-1} = (dZ_l . W_l) * gelu'(Z_{l-1})  (M = bp, N = din_l, K = dout_l)
        Gemm gd = blank(m);
        gd.A = m->dZb[l];
        gd.lda = m->opad[l];
        gd.B = m->WTb[l];
        gd.ldb = m->opad[l];
        gd.M = bp;
        gd.N = m->din[l];
        gd.K = m->opad[l];
        gd.epi = EPI_GELU_GRAD;
        gd.zprev = m->Z[l - 1];
        gd.Z = m->dZ[l - 1];
        gd.ldz = m->dout[l - 1];
        gd.H = m->dZb[l - 1];
        gd.ldh = m->opad[l - 1];
        gd.HT = m->dZT[l - 1];
        gd.ldht = bp;
        if ((rc = gemm(m, gd))) return rc;
    }
    std::vector<double> part(nb + 1);
    MCK(m, cudaMemcpyAsync(part.data(), m->partial, sizeof(double) * nb, cudaMemcpyDeviceToHost, m->stream));
    MCK(m, cudaMemcpyAsync(part.data() + nb, m->msum, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    int rc = check_err(m);
    if (rc) return rc;
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += part[i];
    if (loss) *loss = s / part[nb];
    return LBIF_OK;
}

extern "C" int lbif_mlp_gradients(lbif_mlp m, const float* X, const float* T, const float* mask, int32_t batch,
                                  float* grads, double* loss, int32_t on_device)
{
    if (!m || !X || !T || !mask || batch < 1 || batch > m->max_batch)
        return mfail(m, LBIF_ERR_ARG, "lbif_mlp_gradients: bad arguments");
    int rc = pack_input(m, X, batch, on_device);
    if (rc) return rc;
    if ((rc = forward(m, batch, true))) return rc;
    if ((rc = backward(m, T, mask, batch, on_device, loss))) return rc;
    if (grads) {
        MCK(m, cudaMemcpyAsync(grads, m->g, sizeof(float) * m->nparams,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
        MCK(m, cudaStreamSynchronize(m->stream));
    }
    return LBIF_OK;
}

extern "C" int lbif_mlp_train_step(lbif_mlp m, const float* X, const float* T, const float* mask, int32_t batch,
                                   float lr, float beta1, float beta2, float eps, double* loss, int32_t on_device)
{
    if (!m || !X || !T || !mask || batch < 1 || batch > m->max_batch || !(lr >= 0))
        return mfail(m, LBIF_ERR_ARG, "lbif_mlp_train_step: bad arguments");
    int rc = pack_input(m, X, batch, on_device);
    if (rc) return rc;
    if ((rc = forward(m, batch, true))) return rc;
    if ((rc = backward(m, T, mask, batch, on_device, loss))) return rc;
    m->adam_t += 1;
    const float c1 = (float)(1.0 - pow((double)beta1, (double)m->adam_t));
    const float c2 = (float)(1.0 - pow((double)beta2, (double)m->adam_t));
    k_adam<<<(unsigned)((m->nparams + 255) / 256), 256, 0, m->stream>>>(m->p, m->g, m->m, m->v, m->nparams, lr,
                                                                         beta1, beta2, eps, c1, c2);
    MCK(m, cudaGetLastError());
    if ((rc = refresh_shadows(m))) return rc;
    return LBIF_OK;
}
