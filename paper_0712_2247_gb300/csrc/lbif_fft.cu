// Attractive mean-field tail through the convolution theorem.
//
// The tail force of a node (Sec. Conclusions: a mean-field attraction added
// to the hard-sphere force; Lennard-Jones form with the Barker-Henderson
// split, cut at rcut sigma) is F_att(r)/n0 = n0 m(r) T(r) with m = n/n0 (zero
// outside the fluid) and T(r) = sum_d K(d) m(r + d), K(d) = phi'(|d|) d/|d|
// over sigma <= |d| <= rcut sigma: a correlation of m with a fixed, odd,
// vector kernel. Split m = f + dn with f = 1 on fluid planes and 0 outside:
// the part of f is x,y-uniform, has a z component only,
//   w(z) = sum_dz kappa(dz) f(z + dz),  kappa(dz) = sum_{dx,dy} K_z(dx, dy, dz),
// and is tabulated in double once (it carries the wall attraction; the odd
// kernel cancels it exactly in a periodic box). The small part dn is done in
// the x-y Fourier modes, where the correlation is diagonal; along z it stays
// a short direct sum (walls need no padding):
//   M(k, z)  = FFT_xy[dn(., ., z) f(z)](k)
//   T^(k, z) = sum_dz conj(FFT_xy[K(., ., dz)](k)) M(k, z + dz)
//   T(r)     = IFFT_xy[T^](r) / (nx ny) + (0, 0, w(z))
// The fields are real, so two planes share a complex transform: the forward
// one takes P_j = m(2j) + i m(2j+1) (m = dn f), whose spectrum gives both
// planes' as M(k, 2j) = (P(k) + conj P(-k)) / 2, M(k, 2j+1) = (P(k) -
// conj P(-k)) / 2i; the inverse ones take T_x + i T_y of each plane and
// T_z(2j) + i T_z(2j+1) of each pair. The kernel's transform is computed once
// per handle with the same FFT kernels. The packing of the density rides on
// the first x pass and the product n0 m T on the last one. Cost per step:
// about four passes over a complex field of nx ny nz, instead of ~2 * 10^4
// neighbour reads per node.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "lbif_internal.h"

namespace lbif {
namespace {

constexpr int FFT_THREADS = 256;
constexpr int FFT_GL = 4096;  // lines x line length held by one CTA

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// -i a
__device__ __forceinline__ float2 cmi(float2 a) { return make_float2(a.y, -a.x); }

__device__ __forceinline__ int padded(const Geom& g, int x, int y, int z)
{
    return ((z + g.hw) * g.py + (y + g.hw)) * g.px + (x + g.hw);
}

// Batched Stockham FFT (decimation in frequency, natural order in and out)
// of lines of length L = 2^logL <= 1024 held in shared memory, FFT_GL / L
// lines per CTA. A stage of radix r at stride st (the product of the radices
// before it) maps x_j = X[q + st (p + j M)], M = L / (r st), to
//   Y[q + st (r p + k)] = (sum_j x_j e^{-2 pi i j k / r}) e^{-2 pi i p k st / L};
// radix-4 stages, preceded by one radix-2 stage when logL is odd.
// Along x: line l holds elements l L .. l L + L - 1. Along y: line l = z nx + x
// holds elements z nx L + x + i nx (consecutive lines are consecutive x, so
// the loads and stores of a CTA are row segments of FFT_GL / L nodes).
// tw[j] = exp(-2 pi i j / L) for j < L/2 (copied to shared memory, extended
// by tw[j + L/2] = -tw[j]); inverse = 1 conjugates them (unnormalised).
// Fused ends of the x passes (lines l = j ny + y of a plane-pair field):
// IN reads m(x, y, 2j) + i m(x, y, 2j+1) from the padded density instead of
// `data`; OUT writes Ft = n0 m T of both planes (T_x, T_y from O1, T_z the
// real / imaginary part of the transformed pair) instead of `data`.
struct FftEnds {
    Params P;
    const float* dn;
    const float2* O1;
    const float* w;
    float4* Ft;
};

__device__ __forceinline__ float fluid_dn(const Params& P, const float* dn, int x, int y, int z)
{
    return z < P.g.nz && P.zslit[z] >= 0 ? dn[padded(P.g, x, y, z)] : 0.f;
}

__device__ __forceinline__ void tail_out(const FftEnds& e, int x, int y, int z, float tz)
{
    const Geom& g = e.P.g;
    if (z >= g.nz) return;
    const int s = e.P.zslit[z];
    if (s < 0 || e.P.done[s]) return;
    const float inv = 1.f / ((float)g.nx * (float)g.ny);
    const long long idx = ((long long)z * g.ny + y) * g.nx + x;
    const float pre = e.P.sl[s].rho0 * (1.f + e.dn[padded(g, x, y, z)]);
    const float2 a = e.O1[idx];
    e.Ft[idx] = make_float4(pre * (a.x * inv), pre * (a.y * inv), pre * (tz * inv + e.w[z]), 0.f);
}

template <bool ALONG_Y, bool IN = false, bool OUT = false>
__global__ void __launch_bounds__(FFT_THREADS, 3) k_fft(float2* __restrict__ data, int L, int logL, int lognx,
                                                        long long nlines, const float2* __restrict__ tw, int inverse,
                                                        FftEnds ends)
{
    extern __shared__ float2 fsm[];
    const int G = FFT_GL / L;
    float2* X = fsm;
    float2* Y = fsm + FFT_GL;
    float2* W = fsm + 2 * FFT_GL;  // L twiddles
    const long long l0 = (long long)blockIdx.x * G;
    const int nx = 1 << lognx;
    // element t of the CTA's block (t = g L + i along x, t = i G + g along y):
    // along x the block is contiguous; along y line l0 + g is node column
    // x = (l0 + g) mod nx of plane row z = (l0 + g) / nx (nx a power of two)
    const long long zb = l0 >> lognx;
    const int xb = (int)(l0 & (nx - 1));
    auto addr = [&](int t) -> long long {
        if (ALONG_Y) {
            const int g = t & (G - 1), i = t >> (__ffs(G) - 1);
            const int xg = xb + g;
            return ((zb + (xg >> lognx)) << lognx) * (long long)L + (xg & (nx - 1)) + (long long)i * nx;
        }
        return l0 * L + t;
    };
    auto line = [&](int t) -> long long { return l0 + (ALONG_Y ? (t & (G - 1)) : (t >> logL)); };
    const int half = L >> 1;
    for (int j = threadIdx.x; j < half; j += blockDim.x) {
        float2 w = tw[j];
        if (inverse) w.y = -w.y;
        W[j] = w;
        W[j + half] = make_float2(-w.x, -w.y);
    }
    // G L = FFT_GL: a fixed count of independent loads per thread, all issued
    // before the first store
    constexpr int PT = FFT_GL / FFT_THREADS;
    float2 v[PT];
#pragma unroll
    for (int k = 0; k < PT; ++k) {
        const int t = threadIdx.x + k * FFT_THREADS;
        const long long l = line(t);
        if (IN) {
            const int ny = ends.P.g.ny;
            const int y = (int)(l % ny), j = (int)(l / ny), x = t & (L - 1);
            v[k] = l < nlines ? make_float2(fluid_dn(ends.P, ends.dn, x, y, 2 * j),
                                            fluid_dn(ends.P, ends.dn, x, y, 2 * j + 1))
                              : make_float2(0.f, 0.f);
        } else {
            v[k] = l < nlines ? data[addr(t)] : make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int k = 0; k < PT; ++k) {
        const int t = threadIdx.x + k * FFT_THREADS;
        X[ALONG_Y ? (t & (G - 1)) * L + (t >> (__ffs(G) - 1)) : t] = v[k];
    }
    __syncthreads();
    int st = 1;
    if (logL & 1) {
        // radix 2: M = L / 2
        for (int t = threadIdx.x; t < G * half; t += blockDim.x) {
            const int g = t / half, p = t - g * half;
            const float2 a = X[g * L + p], c = X[g * L + p + half];
            Y[g * L + 2 * p] = cadd(a, c);
            Y[g * L + 2 * p + 1] = cmul(csub(a, c), W[p]);
        }
        __syncthreads();
        float2* tmp = X;
        X = Y;
        Y = tmp;
        st = 2;
    }
    const int quarter = L >> 2;
    for (; st < L; st <<= 2) {
        const int M = L / (4 * st);
        for (int t = threadIdx.x; t < G * quarter; t += blockDim.x) {
            const int g = t / quarter, b = t - g * quarter;
            const int p = b / st, q = b - p * st;
            const float2* xs = X + g * L + q + st * p;
            const float2 x0 = xs[0], x1 = xs[st * M], x2 = xs[2 * st * M], x3 = xs[3 * st * M];
            const float2 t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3);
            const float2 t3 = inverse ? cmi(csub(x3, x1)) : cmi(csub(x1, x3));
            const int e = p * st;  // twiddle exponents e k, k = 1, 2, 3 (all < L)
            float2* ys = Y + g * L + q + 4 * st * p;
            ys[0] = cadd(t0, t2);
            ys[st] = cmul(cadd(t1, t3), W[e]);
            ys[2 * st] = cmul(csub(t0, t2), W[2 * e]);
            ys[3 * st] = cmul(csub(t1, t3), W[3 * e]);
        }
        __syncthreads();
        float2* tmp = X;
        X = Y;
        Y = tmp;
    }
#pragma unroll
    for (int k = 0; k < PT; ++k) {
        const int t = threadIdx.x + k * FFT_THREADS;
        const long long l = line(t);
        if (l >= nlines) continue;
        const float2 r = X[ALONG_Y ? (t & (G - 1)) * L + (t >> (__ffs(G) - 1)) : t];
        if (OUT) {
            const int ny = ends.P.g.ny;
            const int y = (int)(l % ny), j = (int)(l / ny), x = t & (L - 1);
            tail_out(ends, x, y, 2 * j, r.x);
            tail_out(ends, x, y, 2 * j + 1, r.y);
        } else {
            data[addr(t)] = r;
        }
    }
}

// T^(k, z) = sum_dz conj(Kh_c(k, dz)) M(k, z + dz) for 32 modes (one CTA row)
// and a chunk of ZC planes; M (unpacked from the plane-pair transform Pp at
// k and -k) and Kh staged in shared memory. Output O1 = T^_x + i T^_y per
// plane, O2 = T^_z(2j) + i T^_z(2j+1) per plane pair. Planes outside the grid
// read 0 (walls) or their periodic image. T is real, T^(-k) = conj T^(k):
// only the modes with ky <= ny/2 are computed; those with 0 < ky < ny/2 also
// write their mirror -k (rows 0 and ny/2 hold both members of their pairs and
// write only their own mode, so every output has one writer).
constexpr int ZC = 64, ZB = 8;

__global__ void __launch_bounds__(256) k_tail_zconv(const float2* __restrict__ Pp, const float2* __restrict__ Kh,
                                                    float2* __restrict__ O1, float2* __restrict__ O2, int nx,
                                                    int ny, int nz, int D, int zper)
{
    extern __shared__ float2 zsm[];
    float2* slab = zsm;                      // (ZC + 2D) x 32
    float2* kh = zsm + (ZC + 2 * D) * 32;    // (2D + 1) x 3 x 32
    const long long nxy = (long long)nx * ny;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const long long nhalf = (long long)(ny / 2 + 1) * nx;  // modes with ky <= ny/2
    const bool live = (long long)blockIdx.x * 32 + tx < nhalf;
    const long long col = live ? (long long)blockIdx.x * 32 + tx : 0;
    // the mode -k of k = (col mod nx, col / nx)
    const int kx = (int)(col % nx), ky = (int)(col / nx);
    const long long colm = (long long)((ny - ky) % ny) * nx + (nx - kx) % nx;
    const bool mirror = live && ky > 0 && 2 * ky < ny;
    const int z0 = blockIdx.y * ZC;
    for (int r = ty; r < ZC + 2 * D; r += 8) {
        int z = z0 - D + r;
        float2 v = make_float2(0.f, 0.f);
        bool in = true;
        if (zper) {
            z %= nz;
            if (z < 0) z += nz;
        } else {
            in = z >= 0 && z < nz;
        }
        if (in) {
            const long long j = z >> 1;
            const float2 a = Pp[j * nxy + col], b = Pp[j * nxy + colm];
            // M(2j) = (P(k) + conj P(-k)) / 2, M(2j+1) = (P(k) - conj P(-k)) / 2i
            v = (z & 1) ? make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x))
                        : make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
        }
        slab[r * 32 + tx] = v;
    }
    for (int r = ty; r < (2 * D + 1) * 3; r += 8) kh[r * 32 + tx] = Kh[(long long)r * nxy + col];
    __syncthreads();
    for (int zb = ty * ZB; zb < ZC; zb += 8 * ZB) {
        float2 acc[ZB][3];
#pragma unroll
        for (int j = 0; j < ZB; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[j][c] = make_float2(0.f, 0.f);
        for (int d = 0; d <= 2 * D; ++d) {
            float2 k[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) k[c] = kh[(d * 3 + c) * 32 + tx];
#pragma unroll
            for (int j = 0; j < ZB; ++j) {
                const float2 a = slab[(zb + j + d) * 32 + tx];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    // conj(k) * a
                    acc[j][c].x += k[c].x * a.x + k[c].y * a.y;
                    acc[j][c].y += k[c].x * a.y - k[c].y * a.x;
                }
            }
        }
        if (!live) continue;
#pragma unroll
        for (int j = 0; j < ZB; ++j) {
            const int z = z0 + zb + j;
            if (z >= nz) break;
            const float2 a = acc[j][0], b = acc[j][1];
            O1[(long long)z * nxy + col] = make_float2(a.x - b.y, a.y + b.x);  // a + i b
            if (mirror) O1[(long long)z * nxy + colm] = make_float2(a.x + b.y, b.x - a.y);  // conj a + i conj b
        }
#pragma unroll
        for (int j = 0; j < ZB; j += 2) {
            const int z = z0 + zb + j;  // even: ZC, ZB even
            if (z >= nz) break;
            const float2 a = acc[j][2], b = z + 1 < nz ? acc[j + 1][2] : make_float2(0.f, 0.f);
            O2[(long long)(z >> 1) * nxy + col] = make_float2(a.x - b.y, a.y + b.x);
            if (mirror) O2[(long long)(z >> 1) * nxy + colm] = make_float2(a.x + b.y, b.x - a.y);
        }
    }
}

inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

int ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

size_t fft_smem() { return sizeof(float2) * (2 * FFT_GL + 1024); }

// 256-point lines by the four-step split 256 = 16 x 16: a thread holds the
// stride-16 subsequence n = 16 n1 + s of its line, takes the 16-point DFT
// over n1 in registers, multiplies by W_256^(s k1), exchanges through padded
// shared memory (thread k1 then holds k1 of every subsequence) and takes the
// 16-point DFT over the subsequences: X[k1 + 16 k2]. One exchange instead of
// four shared-memory stages. 16 lines per CTA, 16 threads per line; along y
// the 16 threads of a half-warp are 16 consecutive x columns at one y, along
// x 16 consecutive x of one line, so every access is a 128-byte segment.
__device__ __forceinline__ float2 cmi_dir(float2 a, int inverse)
{
    return inverse ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);  // +i a or -i a
}

// in-place 4-point DFT of (x0, x1, x2, x3)
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3, int inverse)
{
    const float2 t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = cmi_dir(csub(x1, x3), inverse);
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

// 16-point DFT of a[0..15] in registers (16 = 4 x 4), natural order out;
// W = exp(-+ 2 pi i j / 256) for j < 256
__device__ __forceinline__ void dft16(float2 (&a)[16], const float2* W, int inverse)
{
    // DFT4 over n1 of a[4 n1 + n2] for each n2, twiddle W_16^(n2 k1)
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        dft4(a[n2], a[4 + n2], a[8 + n2], a[12 + n2], inverse);
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1)
            if (n2) a[4 * k1 + n2] = cmul(a[4 * k1 + n2], W[16 * n2 * k1]);
    }
    // now b[n2][k1] sits in a[4 k1 + n2]; DFT4 over n2 gives A[k1 + 4 k2]
    float2 r[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 x0 = a[4 * k1], x1 = a[4 * k1 + 1], x2 = a[4 * k1 + 2], x3 = a[4 * k1 + 3];
        dft4(x0, x1, x2, x3, inverse);
        r[k1] = x0;
        r[k1 + 4] = x1;
        r[k1 + 8] = x2;
        r[k1 + 12] = x3;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = r[k];
}

template <bool ALONG_Y, bool IN = false, bool OUT = false>
__global__ void __launch_bounds__(256, 3) k_fft256(float2* __restrict__ data, int lognx, long long nlines,
                                                   const float2* __restrict__ tw, int inverse, FftEnds ends)
{
    constexpr int L = 256, G = 16, TP = 16 * 17 + 1;  // padded line stride of the exchange
    __shared__ float2 W[L];
    __shared__ float2 T[G * TP];
    const int tid = threadIdx.x;
    const int g = ALONG_Y ? (tid & 15) : (tid >> 4);
    const int s = ALONG_Y ? (tid >> 4) : (tid & 15);
    const long long l = (long long)blockIdx.x * G + g;
    const bool live = l < nlines;
    const int nx = 1 << lognx;
    auto addr = [&](int i) -> long long {
        if (ALONG_Y) return ((l >> lognx) << lognx) * L + (l & (nx - 1)) + (long long)i * nx;
        return l * L + i;
    };
    for (int j = tid; j < L / 2; j += blockDim.x) {
        float2 w = tw[j];
        if (inverse) w.y = -w.y;
        W[j] = w;
        W[j + L / 2] = make_float2(-w.x, -w.y);
    }
    float2 a[16];
    int yy = 0, jj = 0;
    if (IN || OUT) {
        const int ny = ends.P.g.ny;
        yy = (int)(l % ny);
        jj = (int)(l / ny);
    }
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) {
        const int i = 16 * n1 + s;
        if (!live)
            a[n1] = make_float2(0.f, 0.f);
        else if (IN)
            a[n1] = make_float2(fluid_dn(ends.P, ends.dn, i, yy, 2 * jj), fluid_dn(ends.P, ends.dn, i, yy, 2 * jj + 1));
        else
            a[n1] = data[addr(i)];
    }
    __syncthreads();  // twiddles
    dft16(a, W, inverse);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1)
        if (s) a[k1] = cmul(a[k1], W[s * k1]);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) T[g * TP + s * 17 + k1] = a[k1];
    __syncthreads();
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) a[n2] = T[g * TP + n2 * 17 + s];
    dft16(a, W, inverse);
    if (!live) return;
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
        const int i = s + 16 * k2;
        if (OUT) {
            tail_out(ends, i, yy, 2 * jj, a[k2].x);
            tail_out(ends, i, yy, 2 * jj + 1, a[k2].y);
        } else {
            data[addr(i)] = a[k2];
        }
    }
}

// one batched pass; `ends` selects the fused x-pass variants: 1 = read the
// packed density (IN), 2 = write the tail force (OUT)
cudaError_t fft_pass(float2* data, int L, int nx, long long nlines, bool along_y, const float2* tw, int inverse,
                     cudaStream_t s, int ends_mode = 0, const FftEnds* ends = nullptr)
{
    FftEnds e0;
    const FftEnds& e = ends ? *ends : e0;
    if (L == 256) {
        const unsigned b256 = nblk(nlines, 16);
        const int lnx = ilog2(nx);
        if (along_y)
            k_fft256<true><<<b256, 256, 0, s>>>(data, lnx, nlines, tw, inverse, e);
        else if (ends_mode == 1)
            k_fft256<false, true, false><<<b256, 256, 0, s>>>(data, lnx, nlines, tw, inverse, e);
        else if (ends_mode == 2)
            k_fft256<false, false, true><<<b256, 256, 0, s>>>(data, lnx, nlines, tw, inverse, e);
        else
            k_fft256<false><<<b256, 256, 0, s>>>(data, lnx, nlines, tw, inverse, e);
        return cudaGetLastError();
    }
    const int G = FFT_GL / L;
    const size_t smem = fft_smem();
    const unsigned blocks = nblk(nlines, G);
    if (along_y)
        k_fft<true><<<blocks, FFT_THREADS, smem, s>>>(data, L, ilog2(L), ilog2(nx), nlines, tw, inverse, e);
    else if (ends_mode == 1)
        k_fft<false, true, false><<<blocks, FFT_THREADS, smem, s>>>(data, L, ilog2(L), ilog2(nx), nlines, tw, inverse, e);
    else if (ends_mode == 2)
        k_fft<false, false, true><<<blocks, FFT_THREADS, smem, s>>>(data, L, ilog2(L), ilog2(nx), nlines, tw, inverse, e);
    else
        k_fft<false><<<blocks, FFT_THREADS, smem, s>>>(data, L, ilog2(L), ilog2(nx), nlines, tw, inverse, e);
    return cudaGetLastError();
}

}  // namespace

bool tail_spectral_ok(const Geom& g)
{
    auto pow2 = [](int v) { return v >= 2 && (v & (v - 1)) == 0; };
    return pow2(g.nx) && pow2(g.ny) && g.nx <= 1024 && g.ny <= 1024 && (long long)g.nx * g.ny >= 32;
}

size_t tail_spectral_bytes(const Geom& g, int D)
{
    const size_t nxy = (size_t)g.nx * g.ny;
    return sizeof(float2) * (3 * nxy * (size_t)g.nz + (size_t)(2 * D + 1) * 3 * nxy + g.nx / 2 + g.ny / 2 +
                             (g.nz + 1) / 2);
}

// Layout of the work buffer: A, O1, O2 (nz nx ny complex each), Kh
// ((2D+1) x 3 x ny x nx), the twiddles of nx and of ny, then w (nz floats).
cudaError_t tail_spectral_init(const Geom& g, int D, const int* pdx, const int* pdy, const int* pdz,
                               const float4* K, int npairs, const int* zslit, float2* work, cudaStream_t s)
{
    const long long nxy = (long long)g.nx * g.ny;
    float2* Kh = work + 3 * nxy * g.nz;
    float2* twx = Kh + (long long)(2 * D + 1) * 3 * nxy;
    float2* twy = twx + g.nx / 2;
    std::vector<float2> tx(g.nx / 2), ty(g.ny / 2);
    for (int j = 0; j < g.nx / 2; ++j)
        tx[j] = make_float2((float)cos(-2.0 * M_PI * j / g.nx), (float)sin(-2.0 * M_PI * j / g.nx));
    for (int j = 0; j < g.ny / 2; ++j)
        ty[j] = make_float2((float)cos(-2.0 * M_PI * j / g.ny), (float)sin(-2.0 * M_PI * j / g.ny));
    // the full odd kernel on the periodic x-y grid, one slice per dz and component
    std::vector<float2> host((size_t)(2 * D + 1) * 3 * nxy, make_float2(0.f, 0.f));
    std::vector<double> acc((size_t)(2 * D + 1) * 3 * nxy, 0.0);
    auto put = [&](int dx, int dy, int dz, int c, double v) {
        const int x = ((dx % g.nx) + g.nx) % g.nx, y = ((dy % g.ny) + g.ny) % g.ny;
        acc[((size_t)(dz + D) * 3 + c) * nxy + (size_t)y * g.nx + x] += v;
    };
    for (int k = 0; k < npairs; ++k) {
        const double kv[3] = {K[k].x, K[k].y, K[k].z};
        for (int c = 0; c < 3; ++c) {
            put(pdx[k], pdy[k], pdz[k], c, kv[c]);
            put(-pdx[k], -pdy[k], -pdz[k], c, -kv[c]);
        }
    }
    for (size_t i = 0; i < host.size(); ++i) host[i] = make_float2((float)acc[i], 0.f);
    // w(z): the x,y-uniform response to the fluid indicator, in double
    std::vector<double> kappa(2 * D + 1, 0.0);
    for (int k = 0; k < npairs; ++k) {
        kappa[pdz[k] + D] += K[k].z;
        kappa[-pdz[k] + D] -= K[k].z;
    }
    std::vector<float> wz(g.nz);
    for (int z = 0; z < g.nz; ++z) {
        double a = 0.0;
        for (int d = -D; d <= D; ++d) {
            int zz = z + d;
            if (g.zper) {
                zz %= g.nz;
                if (zz < 0) zz += g.nz;
            } else if (zz < 0 || zz >= g.nz) {
                continue;
            }
            if (zslit[zz] >= 0) a += kappa[d + D];
        }
        wz[z] = (float)a;
    }
    float* wdev = reinterpret_cast<float*>(twy + g.ny / 2);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(twx, tx.data(), sizeof(float2) * tx.size(), cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyAsync(twy, ty.data(), sizeof(float2) * ty.size(), cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyAsync(Kh, host.data(), sizeof(float2) * host.size(), cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyAsync(wdev, wz.data(), sizeof(float) * wz.size(), cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaFuncSetAttribute(k_tail_zconv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(float2) * ((ZC + 2 * D) * 32 + (2 * D + 1) * 3 * 32)))))
        return e;
    if ((e = cudaFuncSetAttribute(k_fft<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem())))
        return e;
    if ((e = cudaFuncSetAttribute(k_fft<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem())))
        return e;
    if ((e = cudaFuncSetAttribute(k_fft<false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)fft_smem())))
        return e;
    if ((e = cudaFuncSetAttribute(k_fft<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)fft_smem())))
        return e;
    const long long slices = (long long)(2 * D + 1) * 3;
    if ((e = fft_pass(Kh, g.nx, g.nx, slices * g.ny, false, twx, 0, s))) return e;
    if ((e = fft_pass(Kh, g.ny, g.nx, slices * g.nx, true, twy, 0, s))) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t launch_tail_spectral(const Params& P, const float* dn, int D, float2* work, float4* Ft, cudaStream_t s)
{
    const Geom& g = P.g;
    const long long nxy = (long long)g.nx * g.ny;
    const int nz2 = (g.nz + 1) / 2;  // plane pairs
    // work: Pp, O2 (nz2 planes each), O1 (nz planes), then Kh and the twiddles
    float2* Pp = work;
    float2* O2 = Pp + nxy * nz2;
    float2* O1 = O2 + nxy * nz2;
    float2* Kh = work + 3 * nxy * g.nz;
    float2* twx = Kh + (long long)(2 * D + 1) * 3 * nxy;
    float2* twy = twx + g.nx / 2;
    const float* w = reinterpret_cast<const float*>(twy + g.ny / 2);
    FftEnds ends{P, dn, O1, w, Ft};
    cudaError_t e;
    if ((e = fft_pass(Pp, g.nx, g.nx, (long long)g.ny * nz2, false, twx, 0, s, 1, &ends))) return e;
    if ((e = fft_pass(Pp, g.ny, g.nx, (long long)g.nx * nz2, true, twy, 0, s))) return e;
    const size_t zs = sizeof(float2) * ((ZC + 2 * D) * 32 + (2 * D + 1) * 3 * 32);
    const long long nhalf = (long long)(g.ny / 2 + 1) * g.nx;
    dim3 grid((unsigned)((nhalf + 31) / 32), (unsigned)((g.nz + ZC - 1) / ZC));
    k_tail_zconv<<<grid, 256, zs, s>>>(Pp, Kh, O1, O2, g.nx, g.ny, g.nz, D, g.zper);
    if ((e = cudaGetLastError())) return e;
    if ((e = fft_pass(O1, g.ny, g.nx, (long long)g.nx * g.nz, true, twy, 1, s))) return e;
    if ((e = fft_pass(O1, g.nx, g.nx, (long long)g.ny * g.nz, false, twx, 1, s))) return e;
    if ((e = fft_pass(O2, g.ny, g.nx, (long long)g.nx * nz2, true, twy, 1, s))) return e;
    return fft_pass(O2, g.nx, g.nx, (long long)g.ny * nz2, false, twx, 1, s, 2, &ends);
}

}  // namespace lbif
