// Device kernels of the hard-sphere lattice Boltzmann step (sm_103a).
//
// Arithmetic is FP32 on small quantities only. Populations are stored
// relative to the node's reference density (see lbif_internal.h), every
// field entering the nonlocal force is a deviation from the uniform state
// (dn = n/n0 - 1, dG = g2 - g2(eta0)), and mirror-image quadrature points are
// combined before they are summed, so a uniform state gives an exactly zero
// force. FP64 appears only in the profile / mass reductions.
#include <string.h>

#include <atomic>
#include <utility>

#include "lbif_internal.h"

namespace lbif {

// D3Q19, antipodes in consecutive pairs (1,2), (3,4), ..., (17,18). The
// components are returned by switches so that, inside unrolled loops, every
// product with a lattice velocity folds to an add, a subtract or nothing.
__device__ __forceinline__ constexpr int kCx(int i)
{
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__device__ __forceinline__ constexpr int kCy(int i)
{
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__device__ __forceinline__ constexpr int kCz(int i)
{
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__device__ __forceinline__ constexpr float kW(int i)
{
    return i == 0 ? 1.f / 3.f : (i <= 6 ? 1.f / 18.f : 1.f / 36.f);
}
// |c_i|^2 (0, 1 or 2 on D3Q19)
__device__ __forceinline__ constexpr int kC2(int i) { return kCx(i) * kCx(i) + kCy(i) * kCy(i) + kCz(i) * kCz(i); }
__device__ __forceinline__ constexpr int opp_of(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

__device__ __forceinline__ float ldp(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldp(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ void stp(float* p, float v) { *p = v; }
__device__ __forceinline__ void stp(__half* p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

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

// node (x, y, z) lies at least hw from every periodic edge: its padded
// field value has no image in the halo
__device__ __forceinline__ bool no_images(const Geom& g, int x, int y, int z)
{
    return x >= g.hw && x < g.nx - g.hw && y >= g.hw && y < g.ny - g.hw &&
           (!g.zper || (z >= g.hw && z < g.nz - g.hw));
}

// Block -> node mapping of the stencil kernels: a CTA covers a TX x TY (x, y)
// tile of one z plane; CTAs are ordered tile-in-group fastest, then z, then
// group, where a group spans about 128 x 128 nodes. The CTAs resident at any
// moment then cover a compact 128 x 128 x ~20 block whose +-sigma stencil
// footprint stays in L2 instead of spanning 2 sigma + 1 full planes.
struct TileMap {
    int tx, ty, tiles_x, tiles_y, gtx, gty, ngx;
    int flat;  // 1: narrow grid, threads run over (x block, y, z) in order
};

__device__ __forceinline__ bool tile_origin(const Geom& g, const TileMap& tm, int& tile_x,
                                            int& tile_y, int& z)
{
    const int per = tm.gtx * tm.gty;
    const int b = blockIdx.x;
    const int tig = b % per;
    const int rest = b / per;
    z = rest % g.nz;
    const int grp = rest / g.nz;
    tile_x = (grp % tm.ngx) * tm.gtx + tig % tm.gtx;
    tile_y = (grp / tm.ngx) * tm.gty + tig / tm.gtx;
    return tile_x < tm.tiles_x && tile_y < tm.tiles_y;
}

static inline TileMap make_tilemap(const Geom& g, int tx, int ty, int group, unsigned& blocks)
{
    TileMap tm;
    tm.tx = tx;
    tm.ty = ty;
    tm.tiles_x = (g.nx + tx - 1) / tx;
    tm.tiles_y = (g.ny + ty - 1) / ty;
    int want_x = (group + tx - 1) / tx, want_y = (group + ty - 1) / ty;
    tm.gtx = tm.tiles_x < want_x ? tm.tiles_x : want_x;
    tm.gty = tm.tiles_y < want_y ? tm.tiles_y : want_y;
    tm.ngx = (tm.tiles_x + tm.gtx - 1) / tm.gtx;
    int ngy = (tm.tiles_y + tm.gty - 1) / tm.gty;
    blocks = (unsigned)tm.gtx * tm.gty * g.nz * tm.ngx * ngy;
    tm.flat = 0;
    return tm;
}

// narrow grids (nx below one tile row): one thread per block of xw x-nodes,
// consecutive threads over x blocks, then y, then z
static inline TileMap make_flatmap(const Geom& g, int xw, int threads, unsigned& blocks)
{
    TileMap tm;
    memset(&tm, 0, sizeof(tm));
    tm.flat = 1;
    tm.tx = (g.nx + xw - 1) / xw;  // x blocks per row
    long long n = (long long)tm.tx * g.ny * g.nz;
    blocks = (unsigned)((n + threads - 1) / threads);
    return tm;
}

__device__ __forceinline__ bool flat_node(const Geom& g, const TileMap& tm, int xw, int& x, int& y, int& z)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long rows = (long long)g.ny * g.nz;
    if (k >= rows * tm.tx) return false;
    int xb = (int)(k % tm.tx);
    long long r = k / tm.tx;
    y = (int)(r % g.ny);
    z = (int)(r / g.ny);
    x = xb * xw;
    return true;
}

// slit of plane z (-1 for a gap plane between stacked slits)
__device__ __forceinline__ int slit_of(const Params& P, int z) { return __ldg(P.zslit + z); }
__device__ __forceinline__ bool frozen(const Params& P, int s) { return __ldg(P.done + s) != 0; }

template <typename T>
__device__ __forceinline__ void load_pops(const Params& P, const T* __restrict__ pop, long long idx,
                                          float h[Q])
{
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = ldp(pop + (long long)i * P.g.Npad + idx);
}

// acc += c x for a lattice-velocity component c in {-1, 0, 1} known after
// unrolling (a product with a zero component is not folded under IEEE rules,
// so the zero case must not be written as one)
__device__ __forceinline__ void add_c(float& acc, int c, float x)
{
    if (c > 0) acc += x;
    if (c < 0) acc -= x;
}

// S = sum_i w_i g_i (density change since the reference), J = sum_i w_i c_i g_i
__device__ __forceinline__ void sums_of(const float g[Q], float& S, float& jx, float& jy, float& jz)
{
    float s = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float wg = kW(i) * g[i];
        s += wg;
        add_c(ax, kCx(i), wg);
        add_c(ay, kCy(i), wg);
        add_c(az, kCz(i), wg);
    }
    S = s;
    jx = ax;
    jy = ay;
    jz = az;
}

// c_i . (x, y, z), adding only the nonzero components (in increasing axis
// order, as the full dot product rounds them)
__device__ __forceinline__ float dot_c(int i, float x, float y, float z)
{
    const int cx = kCx(i), cy = kCy(i), cz = kCz(i);
    if (cx != 0) {
        float r = cx > 0 ? x : -x;
        add_c(r, cy, y);
        add_c(r, cz, z);
        return r;
    }
    if (cy != 0) {
        float r = cy > 0 ? y : -y;
        add_c(r, cz, z);
        return r;
    }
    return cz > 0 ? z : (cz < 0 ? -z : 0.f);
}

// e_i = h_i^eq - dn = (1 + dn)(3 c.u + 9/2 (c.u)^2 - 3/2 u.u)
__device__ __forceinline__ float eq_excess(int i, float opd, float ux, float uy, float uz, float uu)
{
    float cu = dot_c(i, ux, uy, uz);
    return opd * (3.f * cu + 4.5f * cu * cu - 1.5f * uu);
}

// ---------------------------------------------------------------------------
// initialisation and reference-field plumbing
// ---------------------------------------------------------------------------
struct OutsidePlanes {
    float* p[12];
    float v[12];
    int n;
};

__global__ void k_fill_outside(Params P, OutsidePlanes op)
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
    for (int j = 0; j < op.n; ++j) op.p[j][p] = op.v[j];
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

template <typename T>
__global__ void k_init_noise(Params P, T* pop, float* dn, uint64_t seed, double amp, long long offset)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    if (slit_of(P, z) < 0) return;
    uint64_t r = splitmix64(seed ^ (uint64_t)(offset + idx));
    double U = (double)(r >> 11) * (1.0 / 9007199254740992.0);
    // f_i = w_i n0 (1 + xi): reference xi, all stored deviations 0
    float xi = (float)(amp * (2.0 * U - 1.0));
#pragma unroll
    for (int i = 0; i < Q; ++i) stp(pop + (long long)i * P.g.Npad + idx, 0.f);
    for_images(P.g, x, y, z, [&](int p) { dn[p] = xi; });
}

template <typename T>
__global__ void k_init_fields(Params P, T* pop, float* dn, const float* rho, const float* u)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    const int s = slit_of(P, z);
    if (s < 0) return;
    float d = rho[idx] / P.sl[s].rho0 - 1.f;
    float ux = 0.f, uy = 0.f, uz = 0.f;
    if (u) {
        ux = u[idx];
        uy = u[P.g.N + idx];
        uz = u[2 * P.g.N + idx];
    }
    float uu = ux * ux + uy * uy + uz * uz;
    float opd = 1.f + d;
#pragma unroll
    for (int i = 0; i < Q; ++i) stp(pop + (long long)i * P.g.Npad + idx, eq_excess(i, opd, ux, uy, uz, uu));
    for_images(P.g, x, y, z, [&](int p) { dn[p] = d; });
}

// x,y-uniform fields from per-slit profiles n(z), u_x(z) (row s of n_z, ux_z
// holds slit s, entry j its plane zlo + j)
template <typename T>
__global__ void k_init_profiles(Params P, T* pop, float* dn, const float* n_z, const float* ux_z,
                                int hmax)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    const int s = slit_of(P, z);
    if (s < 0) return;
    const int j = z - P.sl[s].zlo;
    const float d = n_z[(long long)s * hmax + j] / P.sl[s].rho0 - 1.f;
    const float ux = ux_z ? ux_z[(long long)s * hmax + j] : 0.f;
    const float uu = ux * ux, opd = 1.f + d;
#pragma unroll
    for (int i = 0; i < Q; ++i) stp(pop + (long long)i * P.g.Npad + idx, eq_excess(i, opd, ux, 0.f, 0.f, uu));
    for_images(P.g, x, y, z, [&](int p) { dn[p] = d; });
}

__global__ void k_write_ref(Params P, const float* ref, float* dn)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    if (slit_of(P, z) < 0) return;
    float v = ref[idx];
    for_images(P.g, x, y, z, [&](int p) { dn[p] = v; });
}

__global__ void k_read_ref(Params P, const float* dn, float* ref)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    ref[idx] = dn[pidx(P.g, x, y, z)];
}

// ---------------------------------------------------------------------------
// step 1: moments (Sec. Theory: n = int f, n u = int v f)
//   reads the reference R = dn(t-1) from dref, writes dn(t) and u
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_moments(Params P, const T* __restrict__ pop,
                                                 const float* dref, float* dnew, float* oux,
                                                 float* ouy, float* ouz, int* status, int skip_done)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    const int s = slit_of(P, z);
    if (s < 0 || (skip_done && frozen(P, s))) return;
    float g[Q];
    load_pops(P, pop, idx, g);
    float R = dref[pidx(P.g, x, y, z)];
    float S, jx, jy, jz;
    sums_of(g, S, jx, jy, jz);
    float dn = R + S;
    float inv = 1.f / (1.f + dn);
    float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    if (!(1.f + dn > 0.f) || !isfinite(dn) || !isfinite(ux + uy + uz)) atomicOr(status, 1);
    auto put = [&](int p) {
        dnew[p] = dn;
        oux[p] = ux;
        ouy[p] = uy;
        ouz[p] = uz;
    };
    if (no_images(P.g, x, y, z))
        put(pidx(P.g, x, y, z));
    else
        for_images(P.g, x, y, z, put);
}

// ---------------------------------------------------------------------------
// step 2: coarse-grained density over the ball |d| <= sigma/2 and the contact
// value g2(etabar) (Sec. Methods, Fischer-Methfessel prescription)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float g2_deviation(const Params& P, float e0, float dnb, bool& bad)
{
    // g2(eta0 (1 + dnb)) - g2(eta0) written so that every term carries
    // Delta = eta0 dnb: (dN D0 - N0 dD) / (D1 D0), D = (1 - eta)^3
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

__host__ __device__ constexpr int cisqrt(int n)
{
    int w = 0;
    while ((w + 1) * (w + 1) <= n) ++w;
    return w;
}

// tile of the z-marching ball kernel: 32 x 16 nodes, 256 threads, each
// thread a column of BALL_YT = 2 nodes in y (measured at sigma = 12 on a
// 512 x 512 x 192 slit: 1 node per thread 0.86 ms, 2 nodes 0.72 ms, 4 nodes
// 0.90 ms, each with its best CTA count)
constexpr int BALL_TX = 32, BALL_YT = 2, BALL_TY = 8 * BALL_YT, BALL_THREADS = 256;


// x halo of the staged plane tile: R rounded up to 4, so that tile rows and
// their global sources are float4-aligned
template <int R>
constexpr int ball_c4() { return (R + 3) / 4 * 4; }

template <int R>
constexpr int ball_smem_floats()
{
    return (BALL_TY + 2 * R) * (BALL_TX + 2 * ball_c4<R>()) + (R + 1) * (BALL_TY + 2 * R) * BALL_TX;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_wait_parity(uint64_t* mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

constexpr long long BALL_WAIT_LIMIT = 1LL << 22;  // try_wait polls; seconds at most

// Self-test of the bounded wait above: the CTA waits on an mbarrier that
// nothing arrives on (its first phase never completes), gives up after
// `polls` polls, records bit 4 of status as the tile kernels do, and returns.
__global__ void k_wait_selftest(long long polls, int* status)
{
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    long long spins = 0;
    bool ok;
    while (!(ok = mbar_wait_parity(&mbar, 0)) && ++spins < polls) {
    }
    if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicOr(status, 4);
}

// does tile row r (relative to a thread's first node row minus R) enter a
// disc sum D_k of any of the thread's BALL_YT nodes with row half-width w?
__host__ __device__ constexpr bool ball_row_used(int R, int r, int w)
{
    for (int j = 0; j < BALL_YT; ++j) {
        const int dy = r - R - j;
        if (dy < -R || dy > R) continue;
        for (int k = 0; k <= R; ++k) {
            const int rem = R * R - k * k - dy * dy;
            if (rem >= 0 && cisqrt(rem) == w) return true;
        }
    }
    return false;
}

// Compile-time expansion of the disc sums of one thread: for every tile row r
// (in increasing order) and half-width w that some D[k][i] uses, one shared
// memory read, added into exactly those D[k][i].
template <int R, int r, int w, int M>
__device__ __forceinline__ void ball_add_one(float v, float (&D)[R + 1][BALL_YT])
{
    constexpr int i = M / (R + 1), k = M % (R + 1);
    constexpr int dy = r - R - i;
    constexpr int rem = R * R - k * k - dy * dy;
    if constexpr (dy >= -R && dy <= R && rem >= 0 && cisqrt(rem) == w) D[k][i] += v;
}

template <int R, int r, int w, int... M>
__device__ __forceinline__ void ball_add_row(float v, float (&D)[R + 1][BALL_YT],
                                             std::integer_sequence<int, M...>)
{
    (ball_add_one<R, r, w, M>(v, D), ...);
}

template <int R, int N>
__device__ __forceinline__ void ball_disc_row(const float* __restrict__ RS, int off, float (&D)[R + 1][BALL_YT])
{
    constexpr int r = N / (R + 1), w = N % (R + 1);
    constexpr int H = BALL_TY + 2 * R;
    if constexpr (ball_row_used(R, r, w)) {
        const float v = RS[(w * H + r) * BALL_TX + off];
        ball_add_row<R, r, w>(v, D, std::make_integer_sequence<int, BALL_YT * (R + 1)>{});
    }
}

// the comma fold runs the rows in increasing order
template <int R, int... N>
__device__ __forceinline__ void ball_disc_rows(const float* __restrict__ RS, int off, float (&D)[R + 1][BALL_YT],
                                               std::integer_sequence<int, N...>)
{
    (ball_disc_row<R, N>(RS, off, D), ...);
}

// Row sums of every half-width 0..R for four adjacent columns per thread,
// from a staged plane tile T (H x W, column C4 + c holds node column c): the
// window sits in registers, additions grow outwards from the centre column.
template <int R>
__device__ __forceinline__ void ball_rowsums(const float* __restrict__ T, float* __restrict__ RS)
{
    constexpr int TX = BALL_TX, TY = BALL_TY;
    constexpr int C4 = ball_c4<R>();
    constexpr int W = TX + 2 * C4, H = TY + 2 * R;
    constexpr int NF = (C4 + R + 7) / 4;  // float4s a 4-column row-sum group reads
    for (int k = threadIdx.x; k < H * (TX / 4); k += blockDim.x) {
        int row = k / (TX / 4), c = 4 * (k - row * (TX / 4));
        const float* tr = T + row * W + c;
        float t[4 * NF];
#pragma unroll
        for (int i = 0; i < NF; ++i) {
            float4 v = *reinterpret_cast<const float4*>(tr + 4 * i);
            t[4 * i] = v.x;
            t[4 * i + 1] = v.y;
            t[4 * i + 2] = v.z;
            t[4 * i + 3] = v.w;
        }
        float s[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) s[j] = t[C4 + j];
        *reinterpret_cast<float4*>(RS + row * TX + c) = make_float4(s[0], s[1], s[2], s[3]);
#pragma unroll
        for (int w = 1; w <= R; ++w) {
#pragma unroll
            for (int j = 0; j < 4; ++j) s[j] += t[C4 + j - w] + t[C4 + j + w];
            *reinterpret_cast<float4*>(RS + (w * H + row) * TX + c) = make_float4(s[0], s[1], s[2], s[3]);
        }
    }
}

// Disc sums of input plane zi for the thread's BALL_YT nodes, added into the
// register ring acc of the 2R+1 output planes they touch; the completed plane
// zi - R is written (g2 deviation, with its periodic images), the ring shifts.
template <int R>
__device__ __forceinline__ void ball_disc_out(const Params& P, const float* __restrict__ RS,
                                              float (&acc)[2 * R + 1][BALL_YT], int zi, int z0, int x,
                                              int y0, int ty0, int tx, float* __restrict__ dG, int* status,
                                              int skip_done)
{
    constexpr int YT = BALL_YT, TX = BALL_TX;
    const Geom& g = P.g;
    // D[k][i] = sum over dy = -R..R (in that order) of the row sum of
    // half-width cisqrt(R^2 - k^2 - dy^2) at row ty0 + i + dy
    float D[R + 1][YT];
#pragma unroll
    for (int k = 0; k <= R; ++k)
#pragma unroll
        for (int i = 0; i < YT; ++i) D[k][i] = 0.f;
    ball_disc_rows<R>(RS, ty0 * TX + tx, D, std::make_integer_sequence<int, (YT + 2 * R) * (R + 1)>{});
#pragma unroll
    for (int k = 0; k <= R; ++k)
#pragma unroll
        for (int i = 0; i < YT; ++i) {
            acc[R - k][i] += D[k][i];
            if (k) acc[R + k][i] += D[k][i];
        }
    const int zo = zi - R;
    const int so = zo >= z0 ? slit_of(P, zo) : -1;
    if (so >= 0 && x < g.nx && !(skip_done && frozen(P, so))) {
        const float e0 = P.sl[so].eta0;
#pragma unroll
        for (int i = 0; i < YT; ++i) {
            const int y = y0 + ty0 + i;
            if (y >= g.ny) break;
            bool bad;
            float v = g2_deviation(P, e0, acc[0][i] * P.ball_inv, bad);
            if (bad) atomicOr(status, 2);
            if (no_images(g, x, y, zo))
                dG[pidx(g, x, y, zo)] = v;
            else
                for_images(g, x, y, zo, [&](int q) { dG[q] = v; });
        }
    }
#pragma unroll
    for (int j = 0; j < 2 * R; ++j)
#pragma unroll
        for (int i = 0; i < YT; ++i) acc[j][i] = acc[j + 1][i];
#pragma unroll
    for (int i = 0; i < YT; ++i) acc[2 * R][i] = 0.f;
}

// One CTA = a 32 x 16 column of nodes marching up a z chunk. Per input plane:
// stage the plane (+R halo) in shared memory, build x-row sums of every
// half-width 0..R, form the disc sums D_k (disc of radius^2 R^2 - k^2; a
// thread reads each row sum it needs once for its two nodes in y) and add
// them into a register ring of the 2R+1 output planes they touch, emit the
// completed plane.
template <int R>
__global__ void __launch_bounds__(BALL_THREADS) k_ball(Params P, const float* __restrict__ dn,
                                              float* __restrict__ dG, int* status, int zchunk,
                                              int skip_done)
{
    constexpr int TX = BALL_TX, TY = BALL_TY;
    constexpr int C4 = ball_c4<R>();
    constexpr int W = TX + 2 * C4, H = TY + 2 * R;
    extern __shared__ __align__(16) float sm[];
    float* T = sm;           // H x W plane tile
    float* RS = sm + H * W;  // (R+1) x H x TX row sums
    const Geom& g = P.g;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    constexpr int YT = BALL_YT;
    const int tx = threadIdx.x % TX, ty0 = (threadIdx.x / TX) * YT;
    const int x = x0 + tx;
    float acc[2 * R + 1][YT];
#pragma unroll
    for (int j = 0; j <= 2 * R; ++j)
#pragma unroll
        for (int i = 0; i < YT; ++i) acc[j][i] = 0.f;

    for (int zi = z0 - R; zi < z1 + R; ++zi) {
        const float* plane = dn + (long long)(zi + g.hw) * g.py * g.px;
        // stage the plane tile with float4 copies (padded rows are 16-byte
        // aligned and hw >= C4, so every source float4 lies inside its row or
        // entirely past its end)
        for (int k = threadIdx.x; k < H * (W / 4); k += blockDim.x) {
            int row = k / (W / 4), q = k - row * (W / 4);
            int xp = x0 - C4 + g.hw + 4 * q, yp = y0 - R + row + g.hw;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (xp + 3 < g.px && yp < g.py) v = ld4(plane + (long long)yp * g.px + xp);
            *reinterpret_cast<float4*>(T + row * W + 4 * q) = v;
        }
        __syncthreads();
        ball_rowsums<R>(T, RS);
        __syncthreads();
        ball_disc_out<R>(P, RS, acc, zi, z0, x, y0, ty0, tx, dG, status, skip_done);
        __syncthreads();
    }
}

// The same kernel with the plane tiles brought in by the tensor-memory
// accelerator: one cp.async.bulk.tensor copy per plane (a W x H x 1 box of
// the padded density field, out-of-range rows filled with zeros), issued by
// one thread two planes ahead into alternating buffers, completion counted
// in bytes on an mbarrier per buffer. The arithmetic is k_ball's.
template <int R>
__global__ void __launch_bounds__(BALL_THREADS) k_ball_tma(Params P, const __grid_constant__ CUtensorMap tmap,
                                                  float* __restrict__ dG, int* status, int zchunk,
                                                  int skip_done)
{
    constexpr int TX = BALL_TX, TY = BALL_TY;
    constexpr int C4 = ball_c4<R>();
    constexpr int W = TX + 2 * C4, H = TY + 2 * R;
    constexpr int TB = (H * W * 4 + 127) / 128 * 128;  // bytes of one tile buffer
    extern __shared__ __align__(128) unsigned char bsm[];
    float* RS = reinterpret_cast<float*>(bsm + 2 * TB);                 // (R+1) x H x TX
    uint64_t* mbar = reinterpret_cast<uint64_t*>(RS + (R + 1) * H * TX);  // 2 barriers
    const Geom& g = P.g;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    constexpr int YT = BALL_YT;
    const int tx = threadIdx.x % TX, ty0 = (threadIdx.x / TX) * YT;
    const int x = x0 + tx;
    const int np = (z1 + R) - (z0 - R);  // input planes of this chunk
    // box origin in padded coordinates; x0 - C4 + hw is a multiple of 4 (16 bytes)
    const int bx = x0 - C4 + g.hw, by = y0 - R + g.hw;
    if (threadIdx.x == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar + 1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int q) {  // plane z0 - R + q into buffer q & 1 (one thread)
        const int b = q & 1;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar + b)),
                     "r"((uint32_t)(H * W * 4))
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(smem_addr(bsm + b * TB)),
            "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(bx), "r"(by), "r"(z0 - R + q + g.hw), "r"(smem_addr(mbar + b))
            : "memory");
    };
    if (threadIdx.x == 0) {
        issue(0);
        if (np > 1) issue(1);
    }
    float acc[2 * R + 1][YT];
#pragma unroll
    for (int j = 0; j <= 2 * R; ++j)
#pragma unroll
        for (int i = 0; i < YT; ++i) acc[j][i] = 0.f;
    uint32_t pbits = 0u;  // bit b: phase parity expected next on buffer b
    for (int q = 0; q < np; ++q) {
        const int b = q & 1;
        long long spins = 0;
        bool ok;
        while (!(ok = mbar_wait_parity(mbar + b, (pbits >> b) & 1u)) && ++spins < BALL_WAIT_LIMIT) {
        }
        if (!__syncthreads_and(ok)) {
            // record the timeout and wait (bounded) for the copies in flight
            if (threadIdx.x == 0) atomicOr(status, 4);
            for (int k = 0; k < 2; ++k) {
                if (q + k >= np) break;
                const int bk = (q + k) & 1;
                spins = 0;
                while (!mbar_wait_parity(mbar + bk, (pbits >> bk) & 1u) && ++spins < BALL_WAIT_LIMIT) {
                }
            }
            return;
        }
        pbits ^= 1u << b;
        ball_rowsums<R>(reinterpret_cast<const float*>(bsm + b * TB), RS);
        __syncthreads();  // buffer b is read: refill it two planes ahead
        if (threadIdx.x == 0 && q + 2 < np) issue(q + 2);
        ball_disc_out<R>(P, RS, acc, z0 - R + q, z0, x, y0, ty0, tx, dG, status, skip_done);
        __syncthreads();
    }
}

// Narrow grids (a 32 x 8 tile would leave most lanes idle): one thread per
// node, reading the padded field directly. The additions run in the order of
// k_ball (row sums grown outwards from the centre, disc sums over y, then the
// planes in increasing z), so both kernels give bit-identical results.
__global__ void __launch_bounds__(256) k_ball_direct(Params P, const float* __restrict__ dn,
                                                     float* __restrict__ dG, int* status, int skip_done)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    const int so = slit_of(P, z);
    if (so < 0 || (skip_done && frozen(P, so))) return;
    const int R = P.sigma / 2;
    const int p = pidx(P.g, x, y, z);
    float s = 0.f;
    for (int dz = -R; dz <= R; ++dz) {
        float D = 0.f;
        for (int dy = -R; dy <= R; ++dy) {
            const int rem = R * R - dy * dy - dz * dz;
            if (rem < 0) continue;
            const int w = cisqrt(rem);
            const float* row = dn + p + (dz * P.g.py + dy) * P.g.px;
            float r = __ldg(row);
            for (int dx = 1; dx <= w; ++dx) r += __ldg(row - dx) + __ldg(row + dx);
            D += r;
        }
        s += D;
    }
    bool bad;
    float v = g2_deviation(P, P.sl[so].eta0, s * P.ball_inv, bad);
    if (bad) atomicOr(status, 2);
    for_images(P.g, x, y, z, [&](int q) { dG[q] = v; });
}

// ---------------------------------------------------------------------------
// step 3: hard-sphere shell force, Eq. LBHS at constant T, 18-point rule.
//   T_q = A_q - (G0 + A_q) lk s_q.(u_q - u),  A_q = G_q n_q / n0 - G0
//       = G0 dq + gq (1 + dq);  the coupling product is split by axis,
//   T_q = A_q - Pa_q - Pb_q, so that parts that cancel between mirror points
//   cancel exactly before they meet the small remainder.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float shell_A(float dq, float gq, float G0) { return G0 * dq + gq * (1.f + dq); }

template <int A>
__device__ __forceinline__ const float* ufield(const Fields& f)
{
    return A == 0 ? f.ux : (A == 1 ? f.uy : f.uz);
}

// generic path: one node per thread, scalar loads (any even sigma)
template <int A>
__device__ __forceinline__ void axis_pair(const Params& P, const Fields& fl, int p, const float u0[3],
                                          float G0, float lk, float f[3], float* cc)
{
    const int o = P.sh.ax_nb[A], om = P.sh.ax_md[A];
    const float* uf = ufield<A>(fl);
    float dp = __ldg(fl.dn + p + o), dm = __ldg(fl.dn + p - o);
    float up = __ldg(uf + p + o), um = __ldg(uf + p - o);
    float gp = __ldg(fl.dG + p + om), gm = __ldg(fl.dG + p - om);
    float Ap = shell_A(dp, gp, G0), Am = shell_A(dm, gm, G0);
    float tp = Ap - (G0 + Ap) * lk * (up - u0[A]);
    float tm = Am - (G0 + Am) * lk * (u0[A] - um);
    f[A] += (1.f / 30.f) * (tp - tm);
    // Eq. C2eq: sum_q W_q (G_q n_q / n0) s_q.(u_q - u)
    if (cc) *cc += (1.f / 30.f) * ((G0 + Ap) * (up - u0[A]) + (G0 + Am) * (u0[A] - um));
}

template <int PL>
__device__ __forceinline__ void diag_quartet(const Params& P, const Fields& fl, int p,
                                             const float u0[3], float G0, float lk, float f[3], float* cc)
{
    constexpr int a = PL == 2 ? 1 : 0;
    constexpr int b = PL == 0 ? 1 : 2;
    constexpr float h = 0.70710678118654752f;
    const float* fa = a == 0 ? fl.ux : fl.uy;
    const float* fb = b == 1 ? fl.uy : fl.uz;
    // member m: sa = (m & 1) ? -1 : 1, sb = (m & 2) ? -1 : 1
    float dq[4] = {0.f, 0.f, 0.f, 0.f}, ua[4] = {0.f, 0.f, 0.f, 0.f}, ub[4] = {0.f, 0.f, 0.f, 0.f};
    float gq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int oa = P.sh.nb_a[PL][k], ob = P.sh.nb_b[PL][k];
        const int ma = P.sh.md_a[PL][k], mb = P.sh.md_b[PL][k];
        const float w = P.sh.nb_w[PL][k], wm = P.sh.md_w[PL][k];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int sa = (m & 1) ? -1 : 1, sb = (m & 2) ? -1 : 1;
            const int o = p + sa * oa + sb * ob;
            dq[m] = fmaf(w, __ldg(fl.dn + o), dq[m]);
            ua[m] = fmaf(w, __ldg(fa + o), ua[m]);
            ub[m] = fmaf(w, __ldg(fb + o), ub[m]);
            gq[m] = fmaf(wm, __ldg(fl.dG + p + sa * ma + sb * mb), gq[m]);
        }
    }
    float Aq[4], Pa[4], Pb[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float sa = (m & 1) ? -1.f : 1.f, sb = (m & 2) ? -1.f : 1.f;
        Aq[m] = shell_A(dq[m], gq[m], G0);
        float c = (G0 + Aq[m]) * lk * h;
        Pa[m] = c * (sa * (ua[m] - u0[a]));
        Pb[m] = c * (sb * (ub[m] - u0[b]));
    }
    // a-component sums sa T over members paired by equal b offset, b-component sb T
    float da = ((Aq[0] - Aq[1]) - (Pa[0] - Pa[1]) - (Pb[0] - Pb[1])) +
               ((Aq[2] - Aq[3]) - (Pa[2] - Pa[3]) - (Pb[2] - Pb[3]));
    float db = ((Aq[0] - Aq[2]) - (Pa[0] - Pa[2]) - (Pb[0] - Pb[2])) +
               ((Aq[1] - Aq[3]) - (Pa[1] - Pa[3]) - (Pb[1] - Pb[3]));
    f[a] += (h / 15.f) * da;
    f[b] += (h / 15.f) * db;
    if (cc) {
        float t = 0.f;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float sa = (m & 1) ? -1.f : 1.f, sb = (m & 2) ? -1.f : 1.f;
            t += (G0 + Aq[m]) * h * (sa * (ua[m] - u0[a]) + sb * (ub[m] - u0[b]));
        }
        *cc += t / 15.f;
    }
}

__device__ __forceinline__ float coupling_factor(const Params& P, const SlitParam& S, int z)
{
    if (!P.coupling) return 0.f;
    float lam = 1.f;
    if (P.regularize && !P.g.zper) {
        float dw = fminf(z - S.zlo + 0.5f, S.zhi + 0.5f - z);
        lam = 1.f - expf(-dw * P.inv_sigma);
    }
    return lam * P.kappa;
}

// total force F / n0 at a node (body + hard sphere + tail), and the energy
// source of Eq. C2eq over n0 when it is on (0 otherwise)
__device__ __forceinline__ void node_force(const Params& P, const SlitParam& S, const Fields& fl,
                                           const float4* __restrict__ Ft, long long idx, int z,
                                           int p, float& fx, float& fy, float& fz, float& c2)
{
    const float d0 = __ldg(fl.dn + p);
    const float u0[3] = {__ldg(fl.ux + p), __ldg(fl.uy + p), __ldg(fl.uz + p)};
    float opd = 1.f + d0;
    fx = opd * S.body[0];
    fy = opd * S.body[1];
    fz = opd * S.body[2];
    c2 = 0.f;
    if (P.hs) {
        const float lk = coupling_factor(P, S, z);
        const float G0 = S.G0;
        float f[3] = {0.f, 0.f, 0.f};
        float cc = 0.f;
        float* pc = P.c2 ? &cc : nullptr;
        axis_pair<0>(P, fl, p, u0, G0, lk, f, pc);
        axis_pair<1>(P, fl, p, u0, G0, lk, f, pc);
        axis_pair<2>(P, fl, p, u0, G0, lk, f, pc);
        diag_quartet<0>(P, fl, p, u0, G0, lk, f, pc);
        diag_quartet<1>(P, fl, p, u0, G0, lk, f, pc);
        diag_quartet<2>(P, fl, p, u0, G0, lk, f, pc);
        float pre = S.hs_pref * opd;
        fx += pre * f[0];
        fy += pre * f[1];
        fz += pre * f[2];
        // C2 / n0 = -(kT sigma^2 4 pi n0 / 2) (1 + dn) sum_q W_q (G_q n_q / n0) s_q.(u_q - u)
        if (P.c2) c2 = 0.5f * pre * cc;
    }
    if (P.tail) {
        float4 t = Ft[idx];
        fx += t.x;
        fy += t.y;
        fz += t.z;
    }
}

__global__ void __launch_bounds__(256) k_force(Params P, TileMap tm, Fields fl,
                                               const float4* __restrict__ Ft, float4* __restrict__ F)
{
    const Geom& g = P.g;
    int x, y, z;
    if (tm.flat) {
        if (!flat_node(g, tm, 1, x, y, z)) return;
    } else {
        int tx, ty;
        if (!tile_origin(g, tm, tx, ty, z)) return;
        x = tx * tm.tx + threadIdx.x % 32;
        y = ty * tm.ty + threadIdx.x / 32;
        if (x >= g.nx || y >= g.ny) return;
    }
    const int s = slit_of(P, z);
    if (s < 0 || frozen(P, s)) return;
    const long long idx = ((long long)z * g.ny + y) * g.nx + x;
    const SlitParam S = P.sl[s];
    float fx, fy, fz, c2;
    node_force(P, S, fl, Ft, idx, z, pidx(g, x, y, z), fx, fy, fz, c2);
    F[idx] = make_float4(fx, fy, fz, c2);
}

// ---- vectorised path: four consecutive x nodes per thread, float4 loads ----
// (sigma a template parameter, so the x offsets and the window alignments are
// compile-time constants; the y / z strides are runtime)
typedef float v4[4];

__host__ __device__ constexpr int floor4(int d) { return d >= 0 ? (d / 4) * 4 : -(((-d) + 3) / 4) * 4; }

__device__ __forceinline__ void set4(v4 r, float4 a)
{
    r[0] = a.x;
    r[1] = a.y;
    r[2] = a.z;
    r[3] = a.w;
}

// values at x offsets D..D+3 of a float4-aligned base
template <int D>
__device__ __forceinline__ void win(const float* __restrict__ f, int b, v4 r)
{
    constexpr int B4 = floor4(D), RR = D - B4;
    if constexpr (RR == 0) {
        set4(r, ld4(f + b + B4));
    } else {
        const float4 A = ld4(f + b + B4), C = ld4(f + b + B4 + 4);
        const float t[8] = {A.x, A.y, A.z, A.w, C.x, C.y, C.z, C.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) r[j] = t[RR + j];
    }
}

// Lanes of a warp in the tiled mapping: the warp is one y row, lane l holds
// the 4-node block at x0 + 4 l, so the value just past (before) a lane's float4
// is the next (previous) lane's first (last) one. hi / lo: this lane loads it
// itself (the last live lane of the row / the first lane).
struct Lanes {
    bool hi, lo;
};

// windows at x offsets D and D + 1 (the two corners along x), sharing loads.
// With LN the fifth value comes from the neighbouring lane by a shuffle, so a
// window costs the float4's wavefronts only (a strided scalar load costs as
// many again).
template <int D, bool LN>
__device__ __forceinline__ void win2(const float* __restrict__ f, int b, v4 w0, v4 w1, Lanes ln)
{
    constexpr int RR = D - floor4(D);
    if constexpr (RR == 0) {
        const float4 A = ld4(f + b + D);
        float s = 0.f;
        if constexpr (LN) s = __shfl_down_sync(0xffffffffu, A.x, 1);
        if (!LN || ln.hi) s = __ldg(f + b + D + 4);
        set4(w0, A);
        w1[0] = A.y;
        w1[1] = A.z;
        w1[2] = A.w;
        w1[3] = s;
    } else if constexpr (RR == 3) {
        const float4 C = ld4(f + b + D + 1);
        float s = 0.f;
        if constexpr (LN) s = __shfl_up_sync(0xffffffffu, C.w, 1);
        if (!LN || ln.lo) s = __ldg(f + b + D);
        w0[0] = s;
        w0[1] = C.x;
        w0[2] = C.y;
        w0[3] = C.z;
        set4(w1, C);
    } else {
        const float4 A = ld4(f + b + D - RR), C = ld4(f + b + D - RR + 4);
        const float t[8] = {A.x, A.y, A.z, A.w, C.x, C.y, C.z, C.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            w0[j] = t[RR + j];
            w1[j] = t[RR + 1 + j];
        }
    }
}

// x offsets of the two corners of a member with x sign SA: SA > 0: (LO, LO+1),
// SA < 0: (-LO, -LO-1); returns the windows in corner order (ka = 0, 1)
template <int LO, int SA, bool LN>
__device__ __forceinline__ void corners_x(const float* __restrict__ f, int b, v4 c0, v4 c1, Lanes ln)
{
    if constexpr (SA > 0)
        win2<LO, LN>(f, b, c0, c1, ln);
    else
        win2<-LO - 1, LN>(f, b, c1, c0, ln);
}

template <int SIG, int PL, int M, bool LN>
__device__ __forceinline__ void member_x(const Params& P, const Fields& fl, int pb, v4 dq, v4 ua,
                                         v4 ub, v4 gq, Lanes ln)
{
    // PL 0: plane (x, y); PL 1: plane (x, z); a = x
    constexpr int LO = cisqrt(SIG * SIG / 2), LOM = cisqrt((SIG / 2) * (SIG / 2) / 2);
    constexpr int SA = (M & 1) ? -1 : 1, SB = (M & 2) ? -1 : 1;
    const int sbs = PL == 0 ? P.g.px : P.g.px * P.g.py;
    const float* fb = PL == 0 ? fl.uy : fl.uz;
#pragma unroll
    for (int kb = 0; kb < 2; ++kb) {
        const int row = pb + SB * (LO + kb) * sbs;
        const float w0 = P.sh.nb_w[PL][2 * kb], w1 = P.sh.nb_w[PL][2 * kb + 1];
        v4 c0, c1;
        corners_x<LO, SA, LN>(fl.dn, row, c0, c1, ln);
#pragma unroll
        for (int j = 0; j < 4; ++j) dq[j] = fmaf(w1, c1[j], fmaf(w0, c0[j], dq[j]));
        corners_x<LO, SA, LN>(fl.ux, row, c0, c1, ln);
#pragma unroll
        for (int j = 0; j < 4; ++j) ua[j] = fmaf(w1, c1[j], fmaf(w0, c0[j], ua[j]));
        corners_x<LO, SA, LN>(fb, row, c0, c1, ln);
#pragma unroll
        for (int j = 0; j < 4; ++j) ub[j] = fmaf(w1, c1[j], fmaf(w0, c0[j], ub[j]));
        const int mrow = pb + SB * (LOM + kb) * sbs;
        const float v0 = P.sh.md_w[PL][2 * kb], v1 = P.sh.md_w[PL][2 * kb + 1];
        corners_x<LOM, SA, LN>(fl.dG, mrow, c0, c1, ln);
#pragma unroll
        for (int j = 0; j < 4; ++j) gq[j] = fmaf(v1, c1[j], fmaf(v0, c0[j], gq[j]));
    }
}

template <int SIG, int M>
__device__ __forceinline__ void member_yz(const Params& P, const Fields& fl, int pb, v4 dq, v4 ua,
                                          v4 ub, v4 gq)
{
    // plane (y, z): no x offset, every corner is an aligned float4
    constexpr int LO = cisqrt(SIG * SIG / 2), LOM = cisqrt((SIG / 2) * (SIG / 2) / 2);
    constexpr int SA = (M & 1) ? -1 : 1, SB = (M & 2) ? -1 : 1;
    const int sy = P.g.px, sz = P.g.px * P.g.py;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ka = k & 1, kb = k >> 1;
        const int o = pb + SA * (LO + ka) * sy + SB * (LO + kb) * sz;
        const int om = pb + SA * (LOM + ka) * sy + SB * (LOM + kb) * sz;
        const float w = P.sh.nb_w[2][k], wm = P.sh.md_w[2][k];
        v4 d, a, b, gg;
        set4(d, ld4(fl.dn + o));
        set4(a, ld4(fl.uy + o));
        set4(b, ld4(fl.uz + o));
        set4(gg, ld4(fl.dG + om));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            dq[j] = fmaf(w, d[j], dq[j]);
            ua[j] = fmaf(w, a[j], ua[j]);
            ub[j] = fmaf(w, b[j], ub[j]);
            gq[j] = fmaf(wm, gg[j], gq[j]);
        }
    }
}

template <int SIG, int PL, int M, bool C2, bool LN>
__device__ __forceinline__ void member_terms(const Params& P, const Fields& fl, int pb,
                                             const v4 ua0, const v4 ub0, float G0, float lk, v4 Aq,
                                             v4 Pa, v4 Pb, v4 Cq, Lanes ln)
{
    constexpr float h = 0.70710678118654752f;
    constexpr float sa = (M & 1) ? -1.f : 1.f, sb = (M & 2) ? -1.f : 1.f;
    v4 dq, ua, ub, gq;
#pragma unroll
    for (int j = 0; j < 4; ++j) dq[j] = ua[j] = ub[j] = gq[j] = 0.f;
    if constexpr (PL == 2)
        member_yz<SIG, M>(P, fl, pb, dq, ua, ub, gq);
    else
        member_x<SIG, PL, M, LN>(P, fl, pb, dq, ua, ub, gq, ln);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        Aq[j] = shell_A(dq[j], gq[j], G0);
        float c = (G0 + Aq[j]) * lk * h;
        Pa[j] = c * (sa * (ua[j] - ua0[j]));
        Pb[j] = c * (sb * (ub[j] - ub0[j]));
        if constexpr (C2) Cq[j] = (G0 + Aq[j]) * h * (sa * (ua[j] - ua0[j]) + sb * (ub[j] - ub0[j]));
    }
}

template <int SIG, int PL, bool C2, bool LN>
__device__ __forceinline__ void quartet4(const Params& P, const Fields& fl, int pb, const v4 u0[3],
                                         float G0, float lk, v4 f[3], v4 cc, Lanes ln)
{
    constexpr int a = PL == 2 ? 1 : 0;
    constexpr int b = PL == 0 ? 1 : 2;
    constexpr float c = 0.70710678118654752f / 15.f;
    v4 A0, P0a, P0b, A1, P1a, P1b, A2, P2a, P2b, A3, P3a, P3b, C0, C1, C2m, C3;
    member_terms<SIG, PL, 0, C2, LN>(P, fl, pb, u0[a], u0[b], G0, lk, A0, P0a, P0b, C0, ln);
    member_terms<SIG, PL, 1, C2, LN>(P, fl, pb, u0[a], u0[b], G0, lk, A1, P1a, P1b, C1, ln);
    member_terms<SIG, PL, 2, C2, LN>(P, fl, pb, u0[a], u0[b], G0, lk, A2, P2a, P2b, C2m, ln);
    member_terms<SIG, PL, 3, C2, LN>(P, fl, pb, u0[a], u0[b], G0, lk, A3, P3a, P3b, C3, ln);
    if constexpr (C2) {
#pragma unroll
        for (int j = 0; j < 4; ++j) cc[j] += (1.f / 15.f) * ((C0[j] + C1[j]) + (C2m[j] + C3[j]));
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float da = ((A0[j] - A1[j]) - (P0a[j] - P1a[j]) - (P0b[j] - P1b[j])) +
                   ((A2[j] - A3[j]) - (P2a[j] - P3a[j]) - (P2b[j] - P3b[j]));
        float db = ((A0[j] - A2[j]) - (P0a[j] - P2a[j]) - (P0b[j] - P2b[j])) +
                   ((A1[j] - A3[j]) - (P1a[j] - P3a[j]) - (P1b[j] - P3b[j]));
        f[a][j] += c * da;
        f[b][j] += c * db;
    }
}

template <int SIG, int A, bool C2>
__device__ __forceinline__ void axis4(const Params& P, const Fields& fl, int pb, const v4 u0[3],
                                      float G0, float lk, v4 f[3], v4 cc)
{
    const float* uf = ufield<A>(fl);
    v4 dp, dm, up, um, gp, gm;
    if constexpr (A == 0) {
        win<SIG>(fl.dn, pb, dp);
        win<-SIG>(fl.dn, pb, dm);
        win<SIG>(uf, pb, up);
        win<-SIG>(uf, pb, um);
        win<SIG / 2>(fl.dG, pb, gp);
        win<-SIG / 2>(fl.dG, pb, gm);
    } else {
        const int st = A == 1 ? P.g.px : P.g.px * P.g.py;
        set4(dp, ld4(fl.dn + pb + SIG * st));
        set4(dm, ld4(fl.dn + pb - SIG * st));
        set4(up, ld4(uf + pb + SIG * st));
        set4(um, ld4(uf + pb - SIG * st));
        set4(gp, ld4(fl.dG + pb + (SIG / 2) * st));
        set4(gm, ld4(fl.dG + pb - (SIG / 2) * st));
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float Ap = shell_A(dp[j], gp[j], G0), Am = shell_A(dm[j], gm[j], G0);
        float tp = Ap - (G0 + Ap) * lk * (up[j] - u0[A][j]);
        float tm = Am - (G0 + Am) * lk * (u0[A][j] - um[j]);
        f[A][j] += (1.f / 30.f) * (tp - tm);
        if constexpr (C2) cc[j] += (1.f / 30.f) * ((G0 + Ap) * (up[j] - u0[A][j]) + (G0 + Am) * (u0[A][j] - um[j]));
    }
}

// At most 128 registers, so that 16 warps share an SM: the kernel waits on
// L1 far more than it computes, and the extra warps hide that latency
// (measured: 146 registers / 12 warps is 6 % slower). CTAs of two warps (a
// 128 x 2 tile), eight per SM (measured at sigma 12 on 512 x 512 x 192:
// 32 / 64 / 128 / 256 / 512 threads 1.658 / 1.610 / 1.631 / 1.705 / 1.820 ms).
// LN: tiled mapping with lane shuffles (every exit above the node's own
// x test is taken by whole warps; lanes past the grid's edge stay, on the
// row's first block, until the stores)
constexpr int FORCE_NT = 64;
template <int SIG, bool C2, bool LN>
__global__ void __launch_bounds__(FORCE_NT, 512 / FORCE_NT) k_force4(Params P, TileMap tm, Fields fl,
                                                const float4* __restrict__ Ft, float4* __restrict__ F)
{
    const Geom& g = P.g;
    int x, y, z;
    bool live = true;
    Lanes ln{false, false};
    if (!LN) {
        if (!flat_node(g, tm, 4, x, y, z)) return;
    } else {
        int tx, ty;
        if (!tile_origin(g, tm, tx, ty, z)) return;
        const int x0 = tx * 128, lane = threadIdx.x % 32;
        x = x0 + 4 * lane;
        y = ty * tm.ty + threadIdx.x / 32;
        if (x0 >= g.nx || y >= g.ny) return;  // whole warp
        live = x < g.nx;
        if (!live) x = x0;
        ln.hi = lane == 31 || x + 4 >= g.nx;
        ln.lo = lane == 0;
    }
    const int s = slit_of(P, z);
    if (s < 0 || frozen(P, s)) return;  // whole warp (one z plane)
    const SlitParam S = P.sl[s];
    const int pb = pidx(g, x, y, z);  // 16-byte aligned: x, hw, px multiples of 4
    v4 d0, u0[3];
    set4(d0, ld4(fl.dn + pb));
    set4(u0[0], ld4(fl.ux + pb));
    set4(u0[1], ld4(fl.uy + pb));
    set4(u0[2], ld4(fl.uz + pb));
    v4 f[3], cc;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < 4; ++j) f[a][j] = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) cc[j] = 0.f;
    if (P.hs) {
        const float lk = coupling_factor(P, S, z);
        axis4<SIG, 0, C2>(P, fl, pb, u0, S.G0, lk, f, cc);
        axis4<SIG, 1, C2>(P, fl, pb, u0, S.G0, lk, f, cc);
        axis4<SIG, 2, C2>(P, fl, pb, u0, S.G0, lk, f, cc);
        quartet4<SIG, 0, C2, LN>(P, fl, pb, u0, S.G0, lk, f, cc, ln);
        quartet4<SIG, 1, C2, LN>(P, fl, pb, u0, S.G0, lk, f, cc, ln);
        quartet4<SIG, 2, C2, LN>(P, fl, pb, u0, S.G0, lk, f, cc, ln);
    }
    if (!live) return;
    const long long idx0 = ((long long)z * g.ny + y) * g.nx + x;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (x + j >= g.nx) break;
        const float opd = 1.f + d0[j];
        const float pre = S.hs_pref * opd;
        float fx = opd * S.body[0] + pre * f[0][j];
        float fy = opd * S.body[1] + pre * f[1][j];
        float fz = opd * S.body[2] + pre * f[2][j];
        if (P.tail) {
            float4 t = Ft[idx0 + j];
            fx += t.x;
            fy += t.y;
            fz += t.z;
        }
        // energy source of Eq. C2eq over n0 (when on)
        const float c2 = C2 && P.hs ? 0.5f * pre * cc[j] : 0.f;
        F[idx0 + j] = make_float4(fx, fy, fz, c2);
    }
}

bool force_vectorised(int sigma) { return sigma == 4 || sigma == 8 || sigma == 12; }

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
    const int s = slit_of(P, z);
    if (s < 0 || frozen(P, s)) return;
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
    float pre = P.sl[s].rho0 * (1.f + __ldg(dn + p));
    Ft[idx] = make_float4(pre * sx, pre * sy, pre * sz, 0.f);
}

// ---------------------------------------------------------------------------
// steps 5-6: BGK collision with the first-order source and push streaming
// with half-way bounce-back (Sec. Methods: forward-Euler update, local
// equilibrium; bounce-back walls). Works on k_i = h_i - dn (populations
// relative to the node's own current density) and stores, at the target,
// the value relative to the target's current density.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256, 4) k_cs(Params P, const T* __restrict__ pin, T* __restrict__ pout,
                                               Fields fl, const float4* __restrict__ F)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    const Geom& g = P.g;
    int x, y, z;
    decompose(g, idx, x, y, z);
    const int s = slit_of(P, z);
    if (s < 0 || frozen(P, s)) return;
    const int zlo = P.sl[s].zlo, zhi = P.sl[s].zhi;
    const float inv_tau = P.sl[s].inv_tau;
    const int p = pidx(g, x, y, z);
    float gi[Q];
    load_pops(P, pin, idx, gi);
    const float d0 = __ldg(fl.dn + p), ux = __ldg(fl.ux + p), uy = __ldg(fl.uy + p),
                uz = __ldg(fl.uz + p);
    const float4 f = __ldg(F + idx);
    float S, jx, jy, jz;
    sums_of(gi, S, jx, jy, jz);
    const float opd = 1.f + d0;
    const float uu = ux * ux + uy * uy + uz * uz;
    const bool interior = x > 0 && x < g.nx - 1 && y > 0 && y < g.ny - 1 && z > zlo && z < zhi;
    if (interior) {
        // no wrap, no wall: target = idx + constant offset. The neighbour
        // densities are fetched together first so their latencies overlap.
        float dd[Q];
        dd[0] = 0.f;
#pragma unroll
        for (int i = 1; i < Q; ++i) dd[i] = __ldg(fl.dn + p + P.nbr[i]);
#pragma unroll
        for (int i = 1; i < Q; ++i) dd[i] = d0 - dd[i];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float k = gi[i] - S;
            float e = eq_excess(i, opd, ux, uy, uz, uu);
            float ks = k - (k - e) * inv_tau + 3.f * dot_c(i, f.x, f.y, f.z) +
                       1.5f * f.w * (float)(kC2(i) - 1);
            stp(pout + (long long)i * g.Npad + (idx + P.soff[i]), ks + dd[i]);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float k = gi[i] - S;
        float e = eq_excess(i, opd, ux, uy, uz, uu);
        float ks = k - (k - e) * inv_tau + 3.f * dot_c(i, f.x, f.y, f.z) +
                       1.5f * f.w * (float)(kC2(i) - 1);
        int tx = x + kCx(i), ty = y + kCy(i), tz = z + kCz(i);
        tx = tx < 0 ? tx + g.nx : (tx >= g.nx ? tx - g.nx : tx);
        ty = ty < 0 ? ty + g.ny : (ty >= g.ny ? ty - g.ny : ty);
        if (g.zper) {
            tz = tz < 0 ? tz + g.nz : (tz >= g.nz ? tz - g.nz : tz);
        } else if (tz < zlo || tz > zhi) {
            stp(pout + (long long)opp_of(i) * g.Npad + idx, ks);
            continue;
        }
        float dt = i == 0 ? d0 : __ldg(fl.dn + p + P.nbr[i]);
        long long t = ((long long)tz * g.ny + ty) * g.nx + tx;
        stp(pout + (long long)i * g.Npad + t, ks + (d0 - dt));
    }
}

// ---------------------------------------------------------------------------
// steps 5-6 fused with step 1 of the next step, in pull form: every node
// gathers the populations that stream into it, applies to each the collision
// of its source node, and forms the new moments from the 19 values it holds,
// so the populations are read and written once per step (push collide-stream
// followed by a moments pass reads them twice). What a source node
// contributes is staged per node in shared memory: a CTA owns a 32 x 4 tile
// of x-y nodes, keeps three planes of it (plus a one-node halo) in a ring,
// and marches up a segment of z planes.
//
// With k_i = h_i - dn (a population relative to its node's current density),
// omega = 1/tau and q = omega (1 + dn), the post-collision value (BGK towards
// the local equilibrium, source 3 c.F + (3/2) F.w (|c|^2 - 1)) is
//   k_i' = (1 - omega) k_i + 3 c.(q u + F) + (9/2) q (c.u)^2 - (3/2) q u.u
//          + (3/2) F.w (|c|^2 - 1),
// which splits by lattice-velocity class into
//   axis a, sign s:            (1 - omega) k + s P_a + C_a
//   plane (a, b), signs sa sb: (1 - omega) k + sa P_a + sb P_b + C_ab + sa sb X_ab
//   rest:                      (1 - omega) k + C_0
// with P = 3 (q u + F), B = K - (3/2) q u.u, C_a = B + (9/2) q u_a^2,
// C_ab = B + (9/2) q (u_a^2 + u_b^2) + (3/2) F.w, X_ab = 9 q u_a u_b and
// C_0 = B - (3/2) F.w = (2 (C_x + C_y + C_z) - (C_xy + C_xz + C_yz)) / 3;
// K = (1 - omega)(R - dn) re-references populations stored relative to R.
// The value reaching r from s = r - c_i, relative to dn(r), is
// k_i'(s) + (dn(s) - dn(r)); at a wall it is k'_{opp i}(r) (half-way
// bounce-back). The new populations are stored relative to the new density
// dn(r) + S, S = sum_i w_i v_i, which is also the next step's reference.
// ---------------------------------------------------------------------------
// 32 x 4 tiles of 128 threads, six CTAs per SM (measured at 512 x 512 x 192, sigma 12, same
// state: 32 x 4 / 128 threads / 6 CTAs 2.186 ms, 32 x 8 / 256 / 3 2.334 ms, 32 x 12 / 384 / 2
// 2.508 ms): more, smaller CTAs keep more population loads in flight across the two barriers
// of each plane
constexpr int CSM_TX = 32, CSM_TY = 4, CSM_THREADS = CSM_TX * CSM_TY;
constexpr int CSM_HX = CSM_TX + 2, CSM_HN = CSM_HX * (CSM_TY + 2);  // staged nodes per plane
// staged quantities: dn, P_x..z, C_x..z, C_xy C_xz C_yz, X_xy X_xz X_yz
constexpr int SQ_DN = 0, SQ_P = 1, SQ_CA = 4, SQ_CP = 7, SQ_X = 10, CSM_NF = 13;
constexpr int CSM_SLOT = CSM_NF * CSM_HN;  // floats per staged plane
size_t csm_smem_bytes() { return sizeof(float) * 3 * CSM_SLOT; }

__device__ __forceinline__ int csm_slot(int q) { return (q + 3) % 3; }

// The halo nodes a thread stages in every plane (NT threads: h = thread,
// thread + NT, ...; at most two): their in-plane padded offset (x, y halo
// images hold the periodic values) and the in-plane index of their periodic
// image in the unpadded force array, or -1 (past the last halo node or a partial
// tile: never gathered).
constexpr int CSM_KS = 2;
struct CsmStaged {
    int p[CSM_KS], n[CSM_KS];
};

template <int NT>
__device__ __forceinline__ CsmStaged csm_staged(const Geom& g, int x0, int y0)
{
    static_assert(NT * CSM_KS >= CSM_HN, "two staged nodes per thread at most");
    CsmStaged st;
#pragma unroll
    for (int k = 0; k < CSM_KS; ++k) {
        const int h = threadIdx.x + k * NT;
        const int X = x0 - 1 + h % CSM_HX, Y = y0 - 1 + h / CSM_HX;
        st.p[k] = st.n[k] = -1;
        if (h >= CSM_HN || X > g.nx || Y > g.ny) continue;
        const int xw = X < 0 ? X + g.nx : (X >= g.nx ? X - g.nx : X);
        const int yw = Y < 0 ? Y + g.ny : (Y >= g.ny ? Y - g.ny : Y);
        st.p[k] = (Y + g.hw) * g.px + (X + g.hw);
        st.n[k] = yw * g.nx + xw;
    }
    return st;
}

// stage plane q (-1 <= q <= nz) of the tile into `slot`
template <int NT>
__device__ __forceinline__ void csm_stage(const Params& P, const CsmIO& io, const float4* __restrict__ F,
                                          float* slot, const CsmStaged& st, int q)
{
    const Geom& g = P.g;
    int zq = q;
    if (g.zper)
        zq = q < 0 ? q + g.nz : (q >= g.nz ? q - g.nz : q);
    else if (q < 0 || q >= g.nz)
        return;  // beyond the walls: only reached through bounce-back
    const int sq = slit_of(P, zq);
    if (sq < 0 || frozen(P, sq)) return;
    const float om = P.sl[sq].inv_tau;
    const int pq = (q + g.hw) * g.py * g.px;
    const float4* Fq = F + (long long)zq * g.ny * g.nx;
#pragma unroll
    for (int k = 0; k < CSM_KS; ++k) {
        if (k * NT >= CSM_HN || st.p[k] < 0) continue;
        const int h = threadIdx.x + k * NT;
        const int p = pq + st.p[k];
        const float4 f = __ldg(Fq + st.n[k]);
        const float d = __ldg(io.dn + p);
        const float ux = __ldg(io.ux + p), uy = __ldg(io.uy + p), uz = __ldg(io.uz + p);
        const float K = io.dref == io.dn ? 0.f : (1.f - om) * (__ldg(io.dref + p) - d);
        const float q1 = om * (1.f + d);
        const float B = K - 1.5f * q1 * (ux * ux + uy * uy + uz * uz);
        const float a = 4.5f * q1, ax = a * ux * ux, ay = a * uy * uy, az = a * uz * uz;
        const float fw = 1.5f * f.w, b = 9.f * q1;
        slot[SQ_DN * CSM_HN + h] = d;
        slot[(SQ_P + 0) * CSM_HN + h] = 3.f * fmaf(q1, ux, f.x);
        slot[(SQ_P + 1) * CSM_HN + h] = 3.f * fmaf(q1, uy, f.y);
        slot[(SQ_P + 2) * CSM_HN + h] = 3.f * fmaf(q1, uz, f.z);
        slot[(SQ_CA + 0) * CSM_HN + h] = B + ax;
        slot[(SQ_CA + 1) * CSM_HN + h] = B + ay;
        slot[(SQ_CA + 2) * CSM_HN + h] = B + az;
        slot[(SQ_CP + 0) * CSM_HN + h] = B + (ax + ay) + fw;
        slot[(SQ_CP + 1) * CSM_HN + h] = B + (ax + az) + fw;
        slot[(SQ_CP + 2) * CSM_HN + h] = B + (ay + az) + fw;
        slot[(SQ_X + 0) * CSM_HN + h] = b * ux * uy;
        slot[(SQ_X + 1) * CSM_HN + h] = b * ux * uz;
        slot[(SQ_X + 2) * CSM_HN + h] = b * uy * uz;
    }
}

// CTAs per SM the register budget is sized for, and z planes per CTA segment
#ifndef CSM_MINB
#define CSM_MINB 6
#endif
#ifndef CSM_LZ
#define CSM_LZ 16
#endif

// the populations of directions [I0, I1) that stream into node (x, y, z):
// v[i - I0]; bit i of bb marks a direction that arrives from a wall
// (bounce-back: the node's own opposite population)
template <int I0, int I1, typename T>
__device__ __forceinline__ void csm_pull(const Params& P, const T* __restrict__ pin, long long idx, int x, int y,
                                         int z, int zlo, int zhi, float* v, unsigned& bb)
{
    const Geom& g = P.g;
    if (x > 0 && x < g.nx - 1 && y > 0 && y < g.ny - 1 && z > zlo && z < zhi) {
#pragma unroll
        for (int i = I0; i < I1; ++i) v[i - I0] = ldp(pin + (long long)i * g.Npad + (idx - P.soff[i]));
        return;
    }
#pragma unroll
    for (int i = I0; i < I1; ++i) {
        int sx = x - kCx(i), sy = y - kCy(i), sz = z - kCz(i);
        sx = sx < 0 ? sx + g.nx : (sx >= g.nx ? sx - g.nx : sx);
        sy = sy < 0 ? sy + g.ny : (sy >= g.ny ? sy - g.ny : sy);
        if (g.zper) {
            sz = sz < 0 ? sz + g.nz : (sz >= g.nz ? sz - g.nz : sz);
        } else if (sz < zlo || sz > zhi) {
            bb |= 1u << i;
            v[i - I0] = ldp(pin + (long long)opp_of(i) * g.Npad + idx);
            continue;
        }
        v[i - I0] = ldp(pin + (long long)i * g.Npad + (((long long)sz * g.ny + sy) * g.nx + sx));
    }
}

// the post-collision values of directions [I0, I1) reaching the node (hc in
// the staged planes), relative to its current density dnr
template <int I0, int I1>
__device__ __forceinline__ void csm_collide(const float* own, const float* below, const float* above, int hc,
                                            float om1, float dnr, unsigned bb, float* v)
{
    constexpr int J0 = I0 == 0 ? 1 : I0;
    if (I0 == 0) {
        const float c0 = (2.f * (own[(SQ_CA + 0) * CSM_HN + hc] + own[(SQ_CA + 1) * CSM_HN + hc] +
                                 own[(SQ_CA + 2) * CSM_HN + hc]) -
                          (own[(SQ_CP + 0) * CSM_HN + hc] + own[(SQ_CP + 1) * CSM_HN + hc] +
                           own[(SQ_CP + 2) * CSM_HN + hc])) * (1.f / 3.f);
        v[0] = fmaf(om1, v[0], c0);
    }
    if (bb == 0) {
        // no wall: every source is r - c_i (offsets fixed at compile time)
#pragma unroll
        for (int i = J0; i < I1; ++i) {
            const int cx = kCx(i), cy = kCy(i), cz = kCz(i);
            const float* sl = (cz > 0 ? below : (cz < 0 ? above : own)) + hc - cx - cy * CSM_HX;
            float t;
            if (kC2(i) == 1) {
                const int a = cx ? 0 : (cy ? 1 : 2);
                const float ca = (float)(cx + cy + cz);
                t = fmaf(ca, sl[(SQ_P + a) * CSM_HN], sl[(SQ_CA + a) * CSM_HN]);
            } else {
                const int pl = cz == 0 ? 0 : (cy == 0 ? 1 : 2);
                const int a = pl == 2 ? 1 : 0, b = pl == 0 ? 1 : 2;
                const float ca = (float)(a == 0 ? cx : cy), cb = (float)(b == 1 ? cy : cz);
                t = sl[(SQ_CP + pl) * CSM_HN] + (ca * sl[(SQ_P + a) * CSM_HN] + cb * sl[(SQ_P + b) * CSM_HN]) +
                    (ca * cb) * sl[(SQ_X + pl) * CSM_HN];
            }
            v[i - I0] = fmaf(om1, v[i - I0], t) + (sl[SQ_DN * CSM_HN] - dnr);
        }
        return;
    }
#pragma unroll
    for (int i = J0; i < I1; ++i) {
        const int cx = kCx(i), cy = kCy(i), cz = kCz(i);
        const bool wall = (bb >> i) & 1u;
        // source node: r - c_i in plane z - c_z, or r itself with -c_i at a wall
        const float* sl = wall ? own : (cz > 0 ? below : (cz < 0 ? above : own));
        const int h = wall ? hc : hc - cx - cy * CSM_HX;
        const float sg = wall ? -1.f : 1.f;
        float t;
        if (kC2(i) == 1) {
            const int a = cx ? 0 : (cy ? 1 : 2);
            const float ca = (float)(cx + cy + cz);
            t = fmaf(sg * ca, sl[(SQ_P + a) * CSM_HN + h], sl[(SQ_CA + a) * CSM_HN + h]);
        } else {
            const int pl = cz == 0 ? 0 : (cy == 0 ? 1 : 2);
            const int a = pl == 2 ? 1 : 0, b = pl == 0 ? 1 : 2;
            const float ca = (float)(a == 0 ? cx : cy), cb = (float)(b == 1 ? cy : cz);
            t = sl[(SQ_CP + pl) * CSM_HN + h] +
                sg * (ca * sl[(SQ_P + a) * CSM_HN + h] + cb * sl[(SQ_P + b) * CSM_HN + h]) +
                (ca * cb) * sl[(SQ_X + pl) * CSM_HN + h];
        }
        const float d = wall ? 0.f : sl[SQ_DN * CSM_HN + h] - dnr;
        v[i - I0] = fmaf(om1, v[i - I0], t) + d;
    }
}

// sum over directions [I0, I1) of w_i v_i and w_i c_i v_i
template <int I0, int I1>
__device__ __forceinline__ void csm_sums(const float* v, float (&m)[4])
{
#pragma unroll
    for (int i = I0; i < I1; ++i) {
        const float wg = kW(i) * v[i - I0];
        m[0] += wg;
        add_c(m[1], kCx(i), wg);
        add_c(m[2], kCy(i), wg);
        add_c(m[3], kCz(i), wg);
    }
}

// one node per thread, a CTA per 32 x 4 tile and z segment (measured: two
// threads per node, each gathering half of the directions and adding the
// partial moments through shared memory, ran slower at twice the warps)
template <typename T>
__global__ void __launch_bounds__(CSM_THREADS, CSM_MINB)
    k_csm(Params P, const T* __restrict__ pin, T* __restrict__ pout, CsmIO io, const float4* __restrict__ F,
          int lz, int tiles_x, int tiles_y, int* status)
{
    constexpr int NT = CSM_THREADS;
    extern __shared__ float sm[];
    const Geom& g = P.g;
    const int tiles = tiles_x * tiles_y;
    const int tile = blockIdx.x % tiles, seg = blockIdx.x / tiles;
    const int x0 = (tile % tiles_x) * CSM_TX, y0 = (tile / tiles_x) * CSM_TY;
    const int t = threadIdx.x;
    const int x = x0 + t % CSM_TX, y = y0 + t / CSM_TX;
    const int hc = (t / CSM_TX + 1) * CSM_HX + t % CSM_TX + 1;
    const bool in_xy = x < g.nx && y < g.ny;
    const int zb = seg * lz, ze = min(zb + lz, g.nz);
    const CsmStaged st = csm_staged<NT>(g, x0, y0);
    csm_stage<NT>(P, io, F, sm + csm_slot(zb - 1) * CSM_SLOT, st, zb - 1);
    csm_stage<NT>(P, io, F, sm + csm_slot(zb) * CSM_SLOT, st, zb);
    for (int z = zb; z < ze; ++z) {
        // issue the population loads first: they do not depend on the ring
        const int s = slit_of(P, z);
        const bool act = in_xy && s >= 0 && !frozen(P, s);
        float v[Q];
        unsigned bb = 0;
        const long long idx = ((long long)z * g.ny + y) * g.nx + x;
        float om = 0.f;
        if (act) {
            const int zlo = P.sl[s].zlo, zhi = P.sl[s].zhi;
            om = P.sl[s].inv_tau;
            csm_pull<0, Q>(P, pin, idx, x, y, z, zlo, zhi, v, bb);
        }
        __syncthreads();  // the slot of plane z - 2 is free
        csm_stage<NT>(P, io, F, sm + csm_slot(z + 1) * CSM_SLOT, st, z + 1);
        __syncthreads();
        float m[4] = {0.f, 0.f, 0.f, 0.f};
        float dnr = 0.f;
        if (act) {
            const float* own = sm + csm_slot(z) * CSM_SLOT;
            const float* below = sm + csm_slot(z - 1) * CSM_SLOT;
            const float* above = sm + csm_slot(z + 1) * CSM_SLOT;
            dnr = own[SQ_DN * CSM_HN + hc];
            csm_collide<0, Q>(own, below, above, hc, 1.f - om, dnr, bb, v);
            csm_sums<0, Q>(v, m);
        }
        if (!act) continue;
        const float S = m[0];
#pragma unroll
        for (int i = 0; i < Q; ++i) stp(pout + (long long)i * g.Npad + idx, v[i] - S);
        const float dn = dnr + S;
        const float inv = 1.f / (1.f + dn);
        const float ux = m[1] * inv, uy = m[2] * inv, uz = m[3] * inv;
        if (!(1.f + dn > 0.f) || !isfinite(dn) || !isfinite(ux + uy + uz)) atomicOr(status, 1);
        auto put = [&](int p) {
            io.dnw[p] = dn;
            io.uxw[p] = ux;
            io.uyw[p] = uy;
            io.uzw[p] = uz;
        };
        if (no_images(g, x, y, z))
            put(pidx(g, x, y, z));
        else
            for_images(g, x, y, z, put);
    }
}

// ---------------------------------------------------------------------------
// outputs
// ---------------------------------------------------------------------------
__global__ void k_force_soa(Params P, const float4* __restrict__ F, float* __restrict__ out)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    float4 v = F[idx];
    out[idx] = v.x;
    out[P.g.N + idx] = v.y;
    out[2 * P.g.N + idx] = v.z;
}

// sum over the 18 points of W_q A_q (A_q = G_q n_q / n0 - G0)
__device__ __forceinline__ float shell_A_sum(const Params& P, const Fields& fl, int p, float G0)
{
    float s = 0.f;
    for (int a = 0; a < 3; ++a)
        for (int sg = -1; sg <= 1; sg += 2) {
            float dq = __ldg(fl.dn + p + sg * P.sh.ax_nb[a]);
            float gq = __ldg(fl.dG + p + sg * P.sh.ax_md[a]);
            s += (1.f / 30.f) * shell_A(dq, gq, G0);
        }
    for (int pl = 0; pl < 3; ++pl)
        for (int m = 0; m < 4; ++m) {
            const int sa = (m & 1) ? -1 : 1, sb = (m & 2) ? -1 : 1;
            float dq = 0.f, gq = 0.f;
            for (int k = 0; k < 4; ++k) {
                dq += P.sh.nb_w[pl][k] * __ldg(fl.dn + p + sa * P.sh.nb_a[pl][k] + sb * P.sh.nb_b[pl][k]);
                gq += P.sh.md_w[pl][k] * __ldg(fl.dG + p + sa * P.sh.md_a[pl][k] + sb * P.sh.md_b[pl][k]);
            }
            s += (1.f / 15.f) * shell_A(dq, gq, G0);
        }
    return s;
}

// rho, u and p = kT n + (kT sigma^3/6) 4 pi n0^2 (1 + dn) sum_q W_q (G0 + A_q)
__global__ void k_moments_out(Params P, Fields fl, float* rho, float* u, float* pr)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    const int sl = slit_of(P, z);
    if (sl < 0) {
        if (rho) rho[idx] = 0.f;
        if (u) u[idx] = u[P.g.N + idx] = u[2 * P.g.N + idx] = 0.f;
        if (pr) pr[idx] = 0.f;
        return;
    }
    const SlitParam S = P.sl[sl];
    int p = pidx(P.g, x, y, z);
    const float d = fl.dn[p];
    if (rho) rho[idx] = S.rho0 * (1.f + d);
    if (u) {
        u[idx] = fl.ux[p];
        u[P.g.N + idx] = fl.uy[p];
        u[2 * P.g.N + idx] = fl.uz[p];
    }
    if (pr) {
        float s = 0.f;
        if (P.hs) s = (S.G0 + shell_A_sum(P, fl, p, S.G0)) * S.p_pref * (1.f + d);
        pr[idx] = (1.f / 3.f) * S.rho0 * (1.f + d) + s;
    }
}

// Per z plane: sum dn, sum ux, sum (1+dn) u (FP64 results, fixed order): CTA
// (z, c) reduces rows [c rc, (c+1) rc) of plane z into part, then
// k_profiles_sum adds the chunks of a plane in order. Per node the work is
// FP32 only (FP64 runs at a small fraction of the FP32 rate on this GPU):
// each thread keeps every sum as an unevaluated pair hi + lo of FP32 numbers,
// updated by Knuth's two-sum, which yields the rounding error of each FP32
// addition exactly, so the pair carries about 48 bits; the products
// (1 + dn) u enter as u + p + e with p = fl(dn u) and e = dn u - p (exact, by
// a fused multiply-add). Each thread converts its pairs to FP64 once; the
// CTA adds them by a fixed FP64 tree.
constexpr int PROF_K = 5;

struct F32Pair {
    float hi, lo;
};

__device__ __forceinline__ void pair_add(F32Pair& a, float x)
{
    const float s = a.hi + x;
    const float bb = s - a.hi;
    a.lo += (a.hi - (s - bb)) + (x - bb);
    a.hi = s;
}

__global__ void k_profiles(Params P, Fields fl, double* part, int chunks)
{
    __shared__ double sh[PROF_K][256];
    const Geom& g = P.g;
    const int z = blockIdx.x, c = blockIdx.y;
    const int rc = (g.ny + chunks - 1) / chunks;
    const int y0 = min(g.ny, c * rc), y1 = min(g.ny, y0 + rc);
    F32Pair a[PROF_K];
#pragma unroll
    for (int j = 0; j < PROF_K; ++j) a[j].hi = a[j].lo = 0.f;
    const int n = (y1 - y0) * g.nx;
    int dy = threadIdx.x / g.nx, x = threadIdx.x - dy * g.nx;
    const int step_y = blockDim.x / g.nx, step_x = blockDim.x - step_y * g.nx;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int p = pidx(g, x, y0 + dy, z);
        const float d = fl.dn[p];
        const float v[3] = {fl.ux[p], fl.uy[p], fl.uz[p]};
        pair_add(a[0], d);
        pair_add(a[1], v[0]);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float pr = d * v[j];
            const float e = fmaf(d, v[j], -pr);
            pair_add(a[2 + j], v[j]);
            pair_add(a[2 + j], pr);
            pair_add(a[2 + j], e);
        }
        // next node of this thread: blockDim.x further in row-major order
        x += step_x;
        dy += step_y;
        if (x >= g.nx) {
            x -= g.nx;
            ++dy;
        }
    }
#pragma unroll
    for (int j = 0; j < PROF_K; ++j) sh[j][threadIdx.x] = (double)a[j].hi + (double)a[j].lo;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int j = 0; j < PROF_K; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < PROF_K) part[((long long)z * chunks + c) * PROF_K + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_profiles_sum(const double* __restrict__ part, int nz, int chunks, double* __restrict__ prof)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)nz * PROF_K) return;
    const long long z = i / PROF_K, j = i - z * PROF_K;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += part[(z * chunks + c) * PROF_K + j];
    prof[i] = s;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline unsigned nblocks(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

cudaError_t launch_fill_outside(const Params& P, float* const* planes, const float* values,
                                int nplanes, cudaStream_t s)
{
    long long total = (long long)P.g.px * P.g.py * 2 * P.g.hw;
    if (P.g.zper || total == 0) return cudaSuccess;
    if (nplanes > 12) return cudaErrorInvalidValue;
    OutsidePlanes op;
    op.n = nplanes;
    for (int j = 0; j < nplanes; ++j) {
        op.p[j] = planes[j];
        op.v[j] = values[j];
    }
    k_fill_outside<<<nblocks(total, 256), 256, 0, s>>>(P, op);
    return cudaGetLastError();
}

cudaError_t launch_init_noise(const Params& P, void* pop, float* dn, uint64_t seed, double amp,
                              long long offset, cudaStream_t s)
{
    if (P.storage == LBIF_STORE_F16)
        k_init_noise<__half><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (__half*)pop, dn, seed, amp, offset);
    else
        k_init_noise<float><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (float*)pop, dn, seed, amp, offset);
    return cudaGetLastError();
}

cudaError_t launch_init_profiles(const Params& P, void* pop, float* dn, const float* n_z,
                                 const float* ux_z, int hmax, cudaStream_t s)
{
    if (P.storage == LBIF_STORE_F16)
        k_init_profiles<__half><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (__half*)pop, dn, n_z, ux_z, hmax);
    else
        k_init_profiles<float><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (float*)pop, dn, n_z, ux_z, hmax);
    return cudaGetLastError();
}

cudaError_t launch_init_fields(const Params& P, void* pop, float* dn, const float* rho,
                               const float* u, cudaStream_t s)
{
    if (P.storage == LBIF_STORE_F16)
        k_init_fields<__half><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (__half*)pop, dn, rho, u);
    else
        k_init_fields<float><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (float*)pop, dn, rho, u);
    return cudaGetLastError();
}

cudaError_t launch_write_ref(const Params& P, const float* ref, float* dn, cudaStream_t s)
{
    k_write_ref<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, ref, dn);
    return cudaGetLastError();
}

cudaError_t launch_read_ref(const Params& P, const float* dn, float* ref, cudaStream_t s)
{
    k_read_ref<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, dn, ref);
    return cudaGetLastError();
}

cudaError_t launch_moments(const Params& P, const void* pop, const float* dref, float* dnew,
                           float* ux, float* uy, float* uz, int* status, int skip_done,
                           cudaStream_t s)
{
    if (P.storage == LBIF_STORE_F16)
        k_moments<__half><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (const __half*)pop, dref, dnew, ux,
                                                               uy, uz, status, skip_done);
    else
        k_moments<float><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (const float*)pop, dref, dnew, ux,
                                                              uy, uz, status, skip_done);
    return cudaGetLastError();
}

template <int R>
static cudaError_t ball_r(const Params& P, const float* dn, float* dG, int* status, int want,
                         int skip_done, const CUtensorMap* tmap, cudaStream_t s)
{
    const Geom& g = P.g;
    constexpr int H = BALL_TY + 2 * R, W = BALL_TX + 2 * ball_c4<R>();
    const size_t smem = tmap ? (size_t)2 * ((H * W * 4 + 127) / 128 * 128) + sizeof(float) * (R + 1) * H * BALL_TX + 16
                             : sizeof(float) * ball_smem_floats<R>();
    // the shared-memory limit is a per-device function attribute: set it
    // once per device that launches the kernel
    static std::atomic<uint64_t> configured{0}, configured_tma{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    std::atomic<uint64_t>& flags = tmap ? configured_tma : configured;
    if (!(flags.load() & bit)) {
        e = tmap ? cudaFuncSetAttribute(k_ball_tma<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                 : cudaFuncSetAttribute(k_ball<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        flags.fetch_or(bit);
    }
    int gx = (g.nx + BALL_TX - 1) / BALL_TX, gy = (g.ny + BALL_TY - 1) / BALL_TY;
    if (want <= 0) want = 608;  // ~4 CTAs per SM on 152 SMs
    int nchunk = (want + gx * gy - 1) / (gx * gy);
    int maxchunk = g.nz / (2 * R) > 1 ? g.nz / (2 * R) : 1;
    if (nchunk > maxchunk) nchunk = maxchunk;
    if (nchunk < 1) nchunk = 1;
    int zchunk = (g.nz + nchunk - 1) / nchunk;
    nchunk = (g.nz + zchunk - 1) / zchunk;
    dim3 grid(gx, gy, nchunk);
    if (tmap)
        k_ball_tma<R><<<grid, BALL_THREADS, smem, s>>>(P, *tmap, dG, status, zchunk, skip_done);
    else
        k_ball<R><<<grid, BALL_THREADS, smem, s>>>(P, dn, dG, status, zchunk, skip_done);
    return cudaGetLastError();
}

void ball_box(int sigma, int* W, int* H)
{
    const int R = sigma / 2;
    *W = BALL_TX + 2 * ((R + 3) / 4 * 4);
    *H = BALL_TY + 2 * R;
}

cudaError_t launch_ball(const Params& P, const float* dn, float* dG, int* status, int want,
                        int skip_done, cudaStream_t s, const CUtensorMap* tmap)
{
    if (P.g.nx < BALL_TX / 2 || P.g.ny < BALL_TY / 2) {
        k_ball_direct<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, dn, dG, status, skip_done);
        return cudaGetLastError();
    }
    switch (P.sigma / 2) {
    case 1: return ball_r<1>(P, dn, dG, status, want, skip_done, tmap, s);
    case 2: return ball_r<2>(P, dn, dG, status, want, skip_done, tmap, s);
    case 3: return ball_r<3>(P, dn, dG, status, want, skip_done, tmap, s);
    case 4: return ball_r<4>(P, dn, dG, status, want, skip_done, tmap, s);
    case 5: return ball_r<5>(P, dn, dG, status, want, skip_done, tmap, s);
    case 6: return ball_r<6>(P, dn, dG, status, want, skip_done, tmap, s);
    case 7: return ball_r<7>(P, dn, dG, status, want, skip_done, tmap, s);
    case 8: return ball_r<8>(P, dn, dG, status, want, skip_done, tmap, s);
    case 9: return ball_r<9>(P, dn, dG, status, want, skip_done, tmap, s);
    case 10: return ball_r<10>(P, dn, dG, status, want, skip_done, tmap, s);
    case 11: return ball_r<11>(P, dn, dG, status, want, skip_done, tmap, s);
    case 12: return ball_r<12>(P, dn, dG, status, want, skip_done, tmap, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tail(const Params& P, const float* dn, const int* off, const float4* K,
                        int npairs, float4* Ft, cudaStream_t s)
{
    k_tail<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, dn, off, K, npairs, Ft);
    return cudaGetLastError();
}

template <int SIG, bool LN>
static void force4_launch(const Params& P, const TileMap& tm, const Fields& f, const float4* Ft, float4* F,
                          unsigned blocks, cudaStream_t s)
{
    if (P.c2)
        k_force4<SIG, true, LN><<<blocks, FORCE_NT, 0, s>>>(P, tm, f, Ft, F);
    else
        k_force4<SIG, false, LN><<<blocks, FORCE_NT, 0, s>>>(P, tm, f, Ft, F);
}

cudaError_t launch_force(const Params& P, const Fields& f, const float4* Ft, float4* F, int group,
                         cudaStream_t s)
{
    unsigned blocks;
    if (group <= 0) group = 128;
    if (force_vectorised(P.sigma)) {
        TileMap tm = P.g.nx < 128 ? make_flatmap(P.g, 4, FORCE_NT, blocks) : make_tilemap(P.g, 128, FORCE_NT / 32, group, blocks);
        switch (P.sigma) {
        case 4:
            if (tm.flat) force4_launch<4, false>(P, tm, f, Ft, F, blocks, s);
            else force4_launch<4, true>(P, tm, f, Ft, F, blocks, s);
            break;
        case 8:
            if (tm.flat) force4_launch<8, false>(P, tm, f, Ft, F, blocks, s);
            else force4_launch<8, true>(P, tm, f, Ft, F, blocks, s);
            break;
        default:
            if (tm.flat) force4_launch<12, false>(P, tm, f, Ft, F, blocks, s);
            else force4_launch<12, true>(P, tm, f, Ft, F, blocks, s);
            break;
        }
    } else {
        TileMap tm = P.g.nx < 32 ? make_flatmap(P.g, 1, 256, blocks) : make_tilemap(P.g, 32, 8, group, blocks);
        k_force<<<blocks, 256, 0, s>>>(P, tm, f, Ft, F);
    }
    return cudaGetLastError();
}

cudaError_t launch_cs(const Params& P, const void* pin, void* pout, const Fields& f,
                      const float4* F, cudaStream_t s)
{
    if (P.storage == LBIF_STORE_F16)
        k_cs<__half><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (const __half*)pin, (__half*)pout, f, F);
    else
        k_cs<float><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (const float*)pin, (float*)pout, f, F);
    return cudaGetLastError();
}

bool csm_ok(const Geom& g) { return g.nx >= CSM_TX && g.ny >= CSM_TY; }

// Measured on GB300 (per-step CUDA-event times, both passes): the fused pass
// wins with FP32 storage on large grids (512x512x192, sigma 12: 2.20 vs
// 2.48 ms with 32 x 4 tiles; with 32 x 8 tiles 2.32 vs 2.52 ms, and 1-3 % at
// 8-12 M nodes) and, with 32 x 8 tiles, lost with FP16 storage (2.69 vs
// 2.26 ms) and on grids too small to fill the GPU with its CTAs
// (256x256x96: 0.61 vs 0.60 ms; 64^3: 0.098 vs 0.060 ms).
bool csm_default(const Geom& g, int storage)
{
    return storage == LBIF_STORE_F32 && csm_ok(g) && g.N >= (1LL << 23);
}

cudaError_t launch_csm(const Params& P, const void* pin, void* pout, const CsmIO& io, const float4* F,
                       int* status, int lz, cudaStream_t s)
{
    const Geom& g = P.g;
    if (lz <= 0) lz = CSM_LZ;
    const int tx = (g.nx + CSM_TX - 1) / CSM_TX, ty = (g.ny + CSM_TY - 1) / CSM_TY;
    const int segs = (g.nz + lz - 1) / lz;
    const long long blocks = (long long)tx * ty * segs;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    const size_t smem = csm_smem_bytes();
    // the shared-memory limit is a per-device function attribute
    static std::atomic<uint64_t> configured{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(k_csm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_csm<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    if (P.storage == LBIF_STORE_F16)
        k_csm<__half><<<(unsigned)blocks, CSM_THREADS, smem, s>>>(P, (const __half*)pin, (__half*)pout, io, F, lz,
                                                                 tx, ty, status);
    else
        k_csm<float><<<(unsigned)blocks, CSM_THREADS, smem, s>>>(P, (const float*)pin, (float*)pout, io, F, lz,
                                                                tx, ty, status);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(long long polls, int* status, cudaStream_t s)
{
    k_wait_selftest<<<1, 128, 0, s>>>(polls, status);
    return cudaGetLastError();
}

cudaError_t launch_force_soa(const Params& P, const float4* F, float* out, cudaStream_t s)
{
    k_force_soa<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, F, out);
    return cudaGetLastError();
}

cudaError_t launch_moments_out(const Params& P, const Fields& f, float* rho, float* u, float* p,
                               cudaStream_t s)
{
    k_moments_out<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, f, rho, u, p);
    return cudaGetLastError();
}

// chunks per plane: enough CTAs to fill the GPU several times over
static int profile_chunks(const Geom& g)
{
    int c = (1216 + g.nz - 1) / g.nz;
    if (c > 32) c = 32;
    if (c > g.ny) c = g.ny;
    return c < 1 ? 1 : c;
}

size_t profile_doubles(const Geom& g) { return (size_t)PROF_K * g.nz * (1 + profile_chunks(g)); }

cudaError_t launch_profiles(const Params& P, const Fields& f, double* prof, cudaStream_t s)
{
    const int chunks = profile_chunks(P.g);
    double* part = prof + (size_t)PROF_K * P.g.nz;
    k_profiles<<<dim3(P.g.nz, chunks), 256, 0, s>>>(P, f, part, chunks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_profiles_sum<<<nblocks((long long)P.g.nz * PROF_K, 256), 256, 0, s>>>(part, P.g.nz, chunks, prof);
    return cudaGetLastError();
}

}  // namespace lbif
