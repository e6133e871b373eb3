// Device kernels of the hard-sphere lattice Boltzmann step (sm_103a).
//
// All arithmetic is FP32 on small quantities: populations are stored as
// relative deviations h_i = f_i/(w_i n0) - 1 and every field that enters the
// nonlocal force is a deviation from the uniform state (dn = n/n0 - 1,
// dG = g2 - g2(eta0)), so the uniform parts cancel exactly instead of being
// subtracted in FP32. FP64 appears only in the profile/mass reductions.
#include "lbif_internal.h"

namespace lbif {

// D3Q19, antipodes in consecutive pairs (1,2), (3,4), ..., (17,18).
__constant__ int kCx[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__constant__ int kCy[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__constant__ int kCz[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
__constant__ float kW[Q] = {1.f / 3.f,  1.f / 18.f, 1.f / 18.f, 1.f / 18.f, 1.f / 18.f,
                            1.f / 18.f, 1.f / 18.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f,
                            1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f,
                            1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f};

__device__ __forceinline__ int opp_of(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

__device__ __forceinline__ float ldp(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldp(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ void stp(float* p, float v) { *p = v; }
__device__ __forceinline__ void stp(__half* p, float v) { *p = __float2half_rn(v); }

__device__ __forceinline__ int pidx(const Geom& g, int x, int y, int z)
{
    return ((z + g.hw) * g.py + (y + g.hw)) * g.px + (x + g.hw);
}

__device__ __forceinline__ void decompose(const Geom& g, long long idx, int& x, int& y, int& z)
{
    int a = (int)(idx / g.nx);
    x = (int)(idx - (long long)a * g.nx);
    z = a / g.ny;
    y = a - z * g.ny;
}

// smallest periodic image x - k n that is >= -hw
__device__ __forceinline__ int img_start(int x, int n, int hw) { return x - ((x + hw) / n) * n; }

// Visit every padded index holding node (x, y, z): itself and its periodic
// images inside the halo (several on grids smaller than the halo).
template <class Fn>
__device__ __forceinline__ void for_images(const Geom& g, int x, int y, int z, Fn fn)
{
    int z0 = g.zper ? img_start(z, g.nz, g.hw) : z;
    int z1 = g.zper ? g.nz + g.hw : z + 1;
    int y0 = img_start(y, g.ny, g.hw);
    int x0 = img_start(x, g.nx, g.hw);
    for (int zi = z0; zi < z1; zi += g.nz)
        for (int yi = y0; yi < g.ny + g.hw; yi += g.ny)
            for (int xi = x0; xi < g.nx + g.hw; xi += g.nx)
                fn(((zi + g.hw) * g.py + (yi + g.hw)) * g.px + (xi + g.hw));
}

template <typename T>
__device__ __forceinline__ void load_pops(const Params& P, const T* __restrict__ pop, long long idx,
                                          float h[Q])
{
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = ldp(pop + (long long)i * P.g.Npad + idx);
}

// dn = sum w h, u = (sum w c h)/(1 + dn)
__device__ __forceinline__ void moments_of(const float h[Q], float& dn, float& ux, float& uy,
                                           float& uz)
{
    float s = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float wh = kW[i] * h[i];
        s += wh;
        jx += kCx[i] * wh;
        jy += kCy[i] * wh;
        jz += kCz[i] * wh;
    }
    float inv = 1.f / (1.f + s);
    dn = s;
    ux = jx * inv;
    uy = jy * inv;
    uz = jz * inv;
}

// ---------------------------------------------------------------------------
// initialisation
// ---------------------------------------------------------------------------
__global__ void k_fill_outside(Params P, float4* M, float* dn, float* dG)
{
    // constant values beyond the walls: n = 0 (dn = -1), u = 0, g2 unused (0)
    const Geom& g = P.g;
    long long plane = (long long)g.px * g.py;
    long long total = plane * 2 * g.hw;
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= total) return;
    long long zl = k / plane;
    long long rem = k - zl * plane;
    int zp = (int)(zl < g.hw ? zl : zl + g.nz);
    long long p = (long long)zp * plane + rem;
    M[p] = make_float4(-1.f, 0.f, 0.f, 0.f);
    dn[p] = -1.f;
    dG[p] = 0.f;
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

template <typename T>
__global__ void k_init_noise(Params P, T* pop, uint64_t seed, double amp, long long offset)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    uint64_t r = splitmix64(seed ^ (uint64_t)(offset + idx));
    double U = (double)(r >> 11) * (1.0 / 9007199254740992.0);
    // f_i = w_i n0 (1 + xi)  ->  h_i = xi for every direction
    float xi = (float)(amp * (2.0 * U - 1.0));
#pragma unroll
    for (int i = 0; i < Q; ++i) stp(pop + (long long)i * P.g.Npad + idx, xi);
}

template <typename T>
__global__ void k_init_fields(Params P, T* pop, const float* rho, const float* u)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    float dn = rho[idx] / P.rho0 - 1.f;
    float ux = 0.f, uy = 0.f, uz = 0.f;
    if (u) {
        ux = u[idx];
        uy = u[P.g.N + idx];
        uz = u[2 * P.g.N + idx];
    }
    float uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float cu = kCx[i] * ux + kCy[i] * uy + kCz[i] * uz;
        float h = dn + (1.f + dn) * (3.f * cu + 4.5f * cu * cu - 1.5f * uu);
        stp(pop + (long long)i * P.g.Npad + idx, h);
    }
}

// ---------------------------------------------------------------------------
// step 1: moments (Sec. Theory: n = int f, n u = int v f)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_moments(Params P, const T* __restrict__ pop, float4* __restrict__ M,
                          float* __restrict__ dnf, int* status)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    float h[Q];
    load_pops(P, pop, idx, h);
    float dn, ux, uy, uz;
    moments_of(h, dn, ux, uy, uz);
    if (!(1.f + dn > 0.f) || !isfinite(dn) || !isfinite(ux + uy + uz)) atomicOr(status, 1);
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    float4 m = make_float4(dn, ux, uy, uz);
    for_images(P.g, x, y, z, [&](int p) {
        M[p] = m;
        dnf[p] = dn;
    });
}

// ---------------------------------------------------------------------------
// step 2: coarse-grained density over the ball of radius sigma/2 and the
// contact value g2(etabar) (Sec. Methods, Fischer-Methfessel prescription)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float g2_deviation(const Params& P, float dnb, bool& bad)
{
    // g2(eta0 (1 + dnb)) - g2(eta0) written so that every term carries
    // Delta = eta0 dnb: (dN D0 - N0 dD) / (D1 D0), D = (1 - eta)^3
    float e0 = P.eta0;
    float d = e0 * dnb;
    float a = 1.f - e0 - d, b = 1.f - e0;
    float N0, dN;
    if (P.g2form == 1) {
        N0 = 1.f - 0.5f * e0;
        dN = -0.5f * d;
    } else {
        N0 = 1.f - 0.5f * e0 + 0.25f * e0 * e0;
        dN = d * (-0.5f + 0.25f * (2.f * e0 + d));
    }
    float dD = -d * (a * a + a * b + b * b);
    float D0 = b * b * b, D1 = a * a * a;
    bad = !(a > 0.f);
    return (dN * D0 - N0 * dD) / (D1 * D0);
}

__global__ void k_ball(Params P, const float* __restrict__ dn, float* __restrict__ dG, int* status)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    int p = pidx(P.g, x, y, z);
    float s = 0.f;
    for (int k = 0; k < P.nseg; ++k) {
        const float* r = dn + p + P.seg_off[k];
        int len = P.seg_len[k];
        for (int j = 0; j < len; ++j) s += __ldg(r + j);
    }
    bool bad;
    float v = g2_deviation(P, s * P.ball_inv, bad);
    if (bad) atomicOr(status, 2);
    for_images(P.g, x, y, z, [&](int q) { dG[q] = v; });
}

// ---------------------------------------------------------------------------
// step 3: hard-sphere shell force, Eq. LBHS at constant T, 18-point rule
// ---------------------------------------------------------------------------
// T_q = (G_q n_q / n0 - G0) - (G_q n_q / n0) lk s_q.(u_q - u)
__device__ __forceinline__ float shell_term(const ShellPoint& s, const float4* __restrict__ M,
                                            const float* __restrict__ dG, int p, float ux,
                                            float uy, float uz, float G0, float lk)
{
    float dq = 0.f, aq = 0.f, bq = 0.f, cq = 0.f;
    for (int c = 0; c < s.nnb; ++c) {
        float4 v = __ldg(M + p + s.nb_off[c]);
        float w = s.nb_w[c];
        dq += w * v.x;
        aq += w * v.y;
        bq += w * v.z;
        cq += w * v.w;
    }
    float gq = 0.f;
    for (int m = 0; m < s.nmd; ++m) gq += s.md_w[m] * __ldg(dG + p + s.md_off[m]);
    float A = G0 * dq + gq * (1.f + dq);
    float su = s.dir[0] * (aq - ux) + s.dir[1] * (bq - uy) + s.dir[2] * (cq - uz);
    return A - (G0 + A) * lk * su;
}

// total force F / n0 at a node (body + hard sphere + tail)
__device__ __forceinline__ void node_force(const Params& P, const float4* __restrict__ M,
                                           const float* __restrict__ dG,
                                           const float4* __restrict__ Ft, long long idx, int z,
                                           int p, float dn, float ux, float uy, float uz,
                                           float& fx, float& fy, float& fz)
{
    float opd = 1.f + dn;
    fx = opd * P.body[0];
    fy = opd * P.body[1];
    fz = opd * P.body[2];
    if (P.hs) {
        float lk = 0.f;
        if (P.coupling) {
            float lam = 1.f;
            if (P.regularize && !P.g.zper) {
                float dw = fminf(z + 0.5f, P.g.nz - 0.5f - z);
                lam = 1.f - expf(-dw * P.inv_sigma);
            }
            lk = lam * P.kappa;
        }
        float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll 1
        for (int q = 0; q < NSHELL; q += 2) {
            float ta = shell_term(P.sp[q], M, dG, p, ux, uy, uz, P.G0, lk);
            float tb = shell_term(P.sp[q + 1], M, dG, p, ux, uy, uz, P.G0, lk);
            float d = P.sp[q].w * (ta - tb);  // antipodal pair, summed first
            sx += P.sp[q].dir[0] * d;
            sy += P.sp[q].dir[1] * d;
            sz += P.sp[q].dir[2] * d;
        }
        float pre = P.hs_pref * opd;
        fx += pre * sx;
        fy += pre * sy;
        fz += pre * sz;
    }
    if (P.tail) {
        float4 t = Ft[idx];
        fx += t.x;
        fy += t.y;
        fz += t.z;
    }
}

// ---------------------------------------------------------------------------
// step 4: mean-field attractive tail, F/n0 = n0 (1 + dn) sum_d dn(r+d) phi'(|d|) d/|d|
// (odd kernel: pairs +-d share one weight)
// ---------------------------------------------------------------------------
__global__ void k_tail(Params P, const float* __restrict__ dn, const int* __restrict__ off,
                       const float4* __restrict__ K, int npairs, float4* __restrict__ Ft)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    int p = pidx(P.g, x, y, z);
    float sx = 0.f, sy = 0.f, sz = 0.f;
    for (int k = 0; k < npairs; ++k) {
        int o = __ldg(off + k);
        float d = __ldg(dn + p + o) - __ldg(dn + p - o);
        float4 kk = __ldg(K + k);
        sx += kk.x * d;
        sy += kk.y * d;
        sz += kk.z * d;
    }
    float pre = P.rho0 * (1.f + __ldg(dn + p));
    Ft[idx] = make_float4(pre * sx, pre * sy, pre * sz, 0.f);
}

// ---------------------------------------------------------------------------
// steps 5-6: BGK collision with the first-order source and push streaming
// with half-way bounce-back (Sec. Methods: forward-Euler update, local
// equilibrium; bounce-back walls)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_fcs(Params P, const T* __restrict__ pin,
                                             T* __restrict__ pout, const float4* __restrict__ M,
                                             const float* __restrict__ dG,
                                             const float4* __restrict__ Ft)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    const Geom& g = P.g;
    int x, y, z;
    decompose(g, idx, x, y, z);
    int p = pidx(g, x, y, z);
    float h[Q];
    load_pops(P, pin, idx, h);
    float dn, ux, uy, uz;
    moments_of(h, dn, ux, uy, uz);
    float fx, fy, fz;
    node_force(P, M, dG, Ft, idx, z, p, dn, ux, uy, uz, fx, fy, fz);

    float opd = 1.f + dn;
    float uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float cu = kCx[i] * ux + kCy[i] * uy + kCz[i] * uz;
        float heq = dn + opd * (3.f * cu + 4.5f * cu * cu - 1.5f * uu);
        float hs = h[i] - (h[i] - heq) * P.inv_tau + 3.f * (kCx[i] * fx + kCy[i] * fy + kCz[i] * fz);
        int tx = x + kCx[i], ty = y + kCy[i], tz = z + kCz[i];
        tx = tx < 0 ? tx + g.nx : (tx >= g.nx ? tx - g.nx : tx);
        ty = ty < 0 ? ty + g.ny : (ty >= g.ny ? ty - g.ny : ty);
        if (g.zper) {
            tz = tz < 0 ? tz + g.nz : (tz >= g.nz ? tz - g.nz : tz);
        } else if (tz < 0 || tz >= g.nz) {
            stp(pout + (long long)opp_of(i) * g.Npad + idx, hs);
            continue;
        }
        long long t = ((long long)tz * g.ny + ty) * g.nx + tx;
        stp(pout + (long long)i * g.Npad + t, hs);
    }
}

// ---------------------------------------------------------------------------
// outputs
// ---------------------------------------------------------------------------
__global__ void k_force_out(Params P, const float4* __restrict__ M, const float* __restrict__ dG,
                            const float4* __restrict__ Ft, float* __restrict__ F)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    int p = pidx(P.g, x, y, z);
    float4 m = M[p];
    float fx, fy, fz;
    node_force(P, M, dG, Ft, idx, z, p, m.x, m.y, m.z, m.w, fx, fy, fz);
    F[idx] = fx;
    F[P.g.N + idx] = fy;
    F[2 * P.g.N + idx] = fz;
}

// rho, u and p = kT n + (kT sigma^3/6) 4 pi n0^2 (1 + dn) sum_q W_q (G0 + A_q)
__global__ void k_moments_out(Params P, const float4* __restrict__ M, const float* __restrict__ dG,
                              float* rho, float* u, float* pr)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    int p = pidx(P.g, x, y, z);
    float4 m = M[p];
    if (rho) rho[idx] = P.rho0 * (1.f + m.x);
    if (u) {
        u[idx] = m.y;
        u[P.g.N + idx] = m.z;
        u[2 * P.g.N + idx] = m.w;
    }
    if (pr) {
        float s = 0.f;
        if (P.hs) {
            for (int q = 0; q < NSHELL; ++q) {
                const ShellPoint& sp = P.sp[q];
                float dq = 0.f, gq = 0.f;
                for (int c = 0; c < sp.nnb; ++c) dq += sp.nb_w[c] * __ldg(&M[p + sp.nb_off[c]].x);
                for (int c = 0; c < sp.nmd; ++c) gq += sp.md_w[c] * __ldg(dG + p + sp.md_off[c]);
                s += sp.w * (P.G0 * dq + gq * (1.f + dq));
            }
            s = (P.G0 + s) * P.p_pref * (1.f + m.x);
        }
        pr[idx] = (1.f / 3.f) * P.rho0 * (1.f + m.x) + s;
    }
}

// per z plane: sum dn, sum ux, sum (1+dn) u  (FP64, fixed-order tree)
constexpr int PROF_K = 5;
__global__ void k_profiles(Params P, const float4* __restrict__ M, double* prof)
{
    __shared__ double sh[PROF_K][256];
    const Geom& g = P.g;
    int z = blockIdx.x;
    double a[PROF_K] = {0, 0, 0, 0, 0};
    int A = g.nx * g.ny;
    for (int k = threadIdx.x; k < A; k += blockDim.x) {
        int y = k / g.nx, x = k - y * g.nx;
        float4 m = M[pidx(g, x, y, z)];
        double opd = 1.0 + (double)m.x;
        a[0] += (double)m.x;
        a[1] += (double)m.y;
        a[2] += opd * m.y;
        a[3] += opd * m.z;
        a[4] += opd * m.w;
    }
    for (int j = 0; j < PROF_K; ++j) sh[j][threadIdx.x] = a[j];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int j = 0; j < PROF_K; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < PROF_K) prof[(long long)z * PROF_K + threadIdx.x] = sh[threadIdx.x][0];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline unsigned nblocks(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

cudaError_t launch_fill_outside(const Params& P, float4* M, float* dn, float* dG, cudaStream_t s)
{
    long long total = (long long)P.g.px * P.g.py * 2 * P.g.hw;
    if (P.g.zper || total == 0) return cudaSuccess;
    k_fill_outside<<<nblocks(total, 256), 256, 0, s>>>(P, M, dn, dG);
    return cudaGetLastError();
}

cudaError_t launch_init_noise(const Params& P, void* pop, uint64_t seed, double amp,
                              long long offset, cudaStream_t s)
{
    if (P.storage == LBIF_STORE_F16)
        k_init_noise<__half><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (__half*)pop, seed, amp, offset);
    else
        k_init_noise<float><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (float*)pop, seed, amp, offset);
    return cudaGetLastError();
}

cudaError_t launch_init_fields(const Params& P, void* pop, const float* rho, const float* u,
                               cudaStream_t s)
{
    if (P.storage == LBIF_STORE_F16)
        k_init_fields<__half><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (__half*)pop, rho, u);
    else
        k_init_fields<float><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (float*)pop, rho, u);
    return cudaGetLastError();
}

cudaError_t launch_moments(const Params& P, const void* pop, float4* M, float* dn, int* status,
                           cudaStream_t s)
{
    if (P.storage == LBIF_STORE_F16)
        k_moments<__half><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (const __half*)pop, M, dn, status);
    else
        k_moments<float><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (const float*)pop, M, dn, status);
    return cudaGetLastError();
}

cudaError_t launch_ball(const Params& P, const float* dn, float* dG, int* status, cudaStream_t s)
{
    k_ball<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, dn, dG, status);
    return cudaGetLastError();
}

cudaError_t launch_tail(const Params& P, const float* dn, const int* off, const float4* K,
                        int npairs, float4* Ft, cudaStream_t s)
{
    k_tail<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, dn, off, K, npairs, Ft);
    return cudaGetLastError();
}

cudaError_t launch_fcs(const Params& P, const void* pin, void* pout, const float4* M,
                       const float* dG, const float4* Ft, cudaStream_t s)
{
    if (P.storage == LBIF_STORE_F16)
        k_fcs<__half><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (const __half*)pin, (__half*)pout, M,
                                                           dG, Ft);
    else
        k_fcs<float><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (const float*)pin, (float*)pout, M, dG,
                                                          Ft);
    return cudaGetLastError();
}

cudaError_t launch_force_out(const Params& P, const float4* M, const float* dG, const float4* Ft,
                             float* F, cudaStream_t s)
{
    k_force_out<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, M, dG, Ft, F);
    return cudaGetLastError();
}

cudaError_t launch_moments_out(const Params& P, const float4* M, const float* dG, float* rho,
                               float* u, float* p, cudaStream_t s)
{
    k_moments_out<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, M, dG, rho, u, p);
    return cudaGetLastError();
}

cudaError_t launch_profiles(const Params& P, const float4* M, double* prof, cudaStream_t s)
{
    k_profiles<<<P.g.nz, 256, 0, s>>>(P, M, prof);
    return cudaGetLastError();
}

}  // namespace lbif
