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
// RAW: a 16-bit population is kept as its bits in the float's register and
// converted at its first use (late_cvt), so that no instruction waits on the
// gather before the work that is meant to hide its latency
template <bool RAW>
__device__ __forceinline__ float ldq(const float* p) { return ldp(p); }
template <bool RAW>
__device__ __forceinline__ float ldq(const __half* p)
{
    if constexpr (RAW)
        return __int_as_float((int)__half_as_ushort(__ldg(p)));
    else
        return ldp(p);
}
__device__ __forceinline__ float late_cvt(float bits) { return __half2float(__ushort_as_half((unsigned short)__float_as_int(bits))); }
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

// Every initial state below is an equilibrium: its stored populations (the
// non-equilibrium parts, see the pull pass) are 0 (the host zeroes the
// population buffer) and its moments are the fields themselves, written with
// their periodic images.
__global__ void k_init_noise(Params P, float* dn, uint64_t seed, double amp, long long offset)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    if (slit_of(P, z) < 0) return;
    uint64_t r = splitmix64(seed ^ (uint64_t)(offset + idx));
    double U = (double)(r >> 11) * (1.0 / 9007199254740992.0);
    // f_i = w_i n0 (1 + xi) = f_i^eq(n0 (1 + xi), 0); u stays 0
    float xi = (float)(amp * (2.0 * U - 1.0));
    for_images(P.g, x, y, z, [&](int p) { dn[p] = xi; });
}

// the equilibrium of given density and velocity fields (u NULL: at rest)
__global__ void k_init_fields(Params P, float* dn, float* ux, float* uy, float* uz, const float* rho, const float* u)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    const int s = slit_of(P, z);
    if (s < 0) return;
    const float d = rho[idx] / P.sl[s].rho0 - 1.f;
    const float vx = u ? u[idx] : 0.f, vy = u ? u[P.g.N + idx] : 0.f, vz = u ? u[2 * P.g.N + idx] : 0.f;
    for_images(P.g, x, y, z, [&](int p) {
        dn[p] = d;
        ux[p] = vx;
        uy[p] = vy;
        uz[p] = vz;
    });
}

// x,y-uniform equilibria from per-slit profiles n(z), u_x(z) (row s of n_z,
// ux_z holds slit s, entry j its plane zlo + j)
__global__ void k_init_profiles(Params P, float* dn, float* ux, float* uy, float* uz, const float* n_z,
                                const float* ux_z, int hmax)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    const int s = slit_of(P, z);
    if (s < 0) return;
    const int j = z - P.sl[s].zlo;
    const float d = n_z[(long long)s * hmax + j] / P.sl[s].rho0 - 1.f;
    const float vx = ux_z ? ux_z[(long long)s * hmax + j] : 0.f;
    for_images(P.g, x, y, z, [&](int p) {
        dn[p] = d;
        ux[p] = vx;
        uy[p] = 0.f;
        uz[p] = 0.f;
    });
}

// ---- populations in place ---------------------------------------------
// One buffer. Direction i of node (x, y, z) of slit s, in the slit's step t,
// sits at storage node
//   ((zb + (z - zlo - t c_iz) mod R) ny + (y - t c_iy) mod ny) nx + (x - t c_ix) mod nx,
// R = the slit's planes plus one ghost plane beyond its walls (none with
// periodic z). The slot a node's pull reads for direction i (its source
// r - c_i at step t) is then the slot it writes (itself at step t + 1); a
// bounce-back reads the node's own slot of the opposite direction at step t,
// which no other node reads or writes in that step, and writes a slot that
// belongs to a ghost-plane node at step t (read by nobody). Every slot is
// therefore read and written by one thread per step. The slit's clock holds
// t mod (nx, ny, R) and advances after every pull pass (not while the slit
// is frozen, so a frozen slit's slots stay where they are).
__device__ __forceinline__ int wrap_lo(int a, int n) { return a < 0 ? a + n : a; }   // a in [-n, n)
__device__ __forceinline__ int wrap_hi(int a, int n) { return a >= n ? a - n : a; }  // a in [0, 2n)

struct IpSlots {
    int x, xm, xp, y, ym, yp, zr, zm, zp;  // the node's coordinates and c_a = +1 (m) / -1 (p) shifted by t + 1
    int tx, ty, tz;                        // t mod (nx, ny, R)
    int zb, R, nx, ny;
    // the slot of direction i of the node at step t + 1 (= of its source at step t)
    __device__ __forceinline__ int slot(int i) const
    {
        const int cx = kCx(i), cy = kCy(i), cz = kCz(i);
        const int xx = cx > 0 ? xm : (cx < 0 ? xp : x);
        const int yy = cy > 0 ? ym : (cy < 0 ? yp : y);
        const int zz = cz > 0 ? zm : (cz < 0 ? zp : zr);
        return ((zb + zz) * ny + yy) * nx + xx;
    }
    // the slot of the node's own direction opp(i) at step t (bounce-back of i)
    __device__ __forceinline__ int wall_slot(int i) const
    {
        const int cx = kCx(i), cy = kCy(i), cz = kCz(i);
        const int xx = cx > 0 ? wrap_hi(x + tx, nx) : (cx < 0 ? wrap_lo(x - tx, nx) : x);
        const int yy = cy > 0 ? wrap_hi(y + ty, ny) : (cy < 0 ? wrap_lo(y - ty, ny) : y);
        const int zz = cz > 0 ? wrap_hi(zr + tz, R) : (cz < 0 ? wrap_lo(zr - tz, R) : zr);
        return ((zb + zz) * ny + yy) * nx + xx;
    }
};

__device__ __forceinline__ IpSlots ip_slots(const Params& P, const SlitParam& S, int s, int x, int y, int z)
{
    const int4 c = __ldg(P.clk + s);
    IpSlots q;
    q.nx = P.g.nx;
    q.ny = P.g.ny;
    q.zb = S.zb;
    q.R = S.R;
    q.tx = c.x;
    q.ty = c.y;
    q.tz = c.z;
    const int sx = wrap_hi(c.x + 1, q.nx), sy = wrap_hi(c.y + 1, q.ny), sz = wrap_hi(c.z + 1, q.R);
    q.x = x;
    q.xm = wrap_lo(x - sx, q.nx);
    q.xp = wrap_hi(x + sx, q.nx);
    q.y = y;
    q.ym = wrap_lo(y - sy, q.ny);
    q.yp = wrap_hi(y + sy, q.ny);
    q.zr = z - S.zlo;
    q.zm = wrap_lo(q.zr - sz, q.R);
    q.zp = wrap_hi(q.zr + sz, q.R);
    return q;
}

__global__ void k_tick(Params P, int4* clk)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P.nslits || frozen(P, s)) return;
    int4 c = clk[s];
    c.x = c.x + 1 == P.g.nx ? 0 : c.x + 1;
    c.y = c.y + 1 == P.g.ny ? 0 : c.y + 1;
    c.z = c.z + 1 == P.sl[s].R ? 0 : c.z + 1;
    clk[s] = c;
}

// direction i of the current state in node order (gap planes skipped):
// to_pop = 0 gathers it from the buffer into canon, 1 scatters canon into it
template <typename T>
__global__ void k_pop_canon(Params P, T* pop, int i, T* canon, int to_pop)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    const int s = slit_of(P, z);
    if (s < 0) return;
    long long at = idx;
    if (P.inplace) {
        // f_i(r, t) sits at the slot of coordinates r - t c_i
        const SlitParam S = P.sl[s];
        const int4 c = P.clk[s];
        const int xx = kCx(i) > 0 ? wrap_lo(x - c.x, P.g.nx) : (kCx(i) < 0 ? wrap_hi(x + c.x, P.g.nx) : x);
        const int yy = kCy(i) > 0 ? wrap_lo(y - c.y, P.g.ny) : (kCy(i) < 0 ? wrap_hi(y + c.y, P.g.ny) : y);
        const int zr = z - S.zlo;
        const int zz = kCz(i) > 0 ? wrap_lo(zr - c.z, S.R) : (kCz(i) < 0 ? wrap_hi(zr + c.z, S.R) : zr);
        at = ((long long)(S.zb + zz) * P.g.ny + yy) * P.g.nx + xx;
    }
    T* q = pop + (long long)i * P.g.Npad + at;
    if (to_pop)
        *q = canon[idx];
    else
        canon[idx] = *q;
}

// moment fields dn, ux, uy, uz <-> four unpadded N-arrays (checkpoints)
__global__ void k_write_fields(Params P, const float* src, float* dn, float* ux, float* uy, float* uz)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    if (slit_of(P, z) < 0) return;
    const long long N = P.g.N;
    const float a = src[idx], b = src[N + idx], c = src[2 * N + idx], d = src[3 * N + idx];
    for_images(P.g, x, y, z, [&](int p) {
        dn[p] = a;
        ux[p] = b;
        uy[p] = c;
        uz[p] = d;
    });
}

__global__ void k_read_fields(Params P, const float* dn, const float* ux, const float* uy, const float* uz,
                              float* out)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    int x, y, z;
    decompose(P.g, idx, x, y, z);
    const int p = pidx(P.g, x, y, z);
    const long long N = P.g.N;
    out[idx] = dn[p];
    out[N + idx] = ux[p];
    out[2 * N + idx] = uy[p];
    out[3 * N + idx] = uz[p];
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
// 0.90 ms, each with its best CTA count; with tensor-memory-accelerator
// staging, CTAs of 4 / 8 / 16 warps 0.567 / 0.552 / 0.573 ms)
#ifndef BALL_WARPS
#define BALL_WARPS 8
#endif
constexpr int BALL_TX = 32, BALL_YT = 2, BALL_TY = BALL_WARPS * BALL_YT, BALL_THREADS = 32 * BALL_WARPS;


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

// generic path: one node per thread, scalar loads (any even sigma). The x and
// y components are formed from accurate mirror differences as in the
// vectorised path below (see there).
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
    const float DA = A == 2 ? Ap - Am : fmaf(G0, dp - dm, fmaf(gp - gm, 1.f + dp, gm * (dp - dm)));
    f[A] += (1.f / 30.f) * (DA - lk * ((G0 + Ap) * (up - u0[A]) - (G0 + Am) * (u0[A] - um)));
    // Eq. C2eq: sum_q W_q (G_q n_q / n0) s_q.(u_q - u)
    if (cc) *cc += (1.f / 30.f) * ((G0 + Ap) * (up - u0[A]) + (G0 + Am) * (u0[A] - um));
}

template <int PL>
__device__ __forceinline__ void diag_quartet(const Params& P, const Fields& fl, int p, const float u0[3],
                                             float G0, float lk, float f[3], float* cc)
{
    constexpr int a = PL == 2 ? 1 : 0;
    constexpr int b = PL == 0 ? 1 : 2;
    constexpr float h = 0.70710678118654752f;
    const float* fa = a == 0 ? fl.ux : fl.uy;
    const float* fb = b == 1 ? fl.uy : fl.uz;
    // corner values of member m (sa = (m & 1) ? -1 : 1, sb = (m & 2) ? -1 : 1)
    auto nb = [&](int m, int k) { return p + ((m & 1) ? -1 : 1) * P.sh.nb_a[PL][k] + ((m & 2) ? -1 : 1) * P.sh.nb_b[PL][k]; };
    auto md = [&](int m, int k) { return p + ((m & 1) ? -1 : 1) * P.sh.md_a[PL][k] + ((m & 2) ? -1 : 1) * P.sh.md_b[PL][k]; };
    if constexpr (PL == 0) {
        // relative to the node's own n and g2: every member a small deviation
        const float d0 = __ldg(fl.dn + p), g0 = __ldg(fl.dG + p);
        const float Aref = fmaf(G0, d0, g0 * (1.f + d0));
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float sa = (m & 1) ? -1.f : 1.f, sb = (m & 2) ? -1.f : 1.f;
            float dl = 0.f, gl = 0.f, ua = 0.f, ub = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float w = P.sh.nb_w[PL][k], wm = P.sh.md_w[PL][k];
                dl = fmaf(w, __ldg(fl.dn + nb(m, k)) - d0, dl);
                ua = fmaf(w, __ldg(fa + nb(m, k)), ua);
                ub = fmaf(w, __ldg(fb + nb(m, k)), ub);
                gl = fmaf(wm, __ldg(fl.dG + md(m, k)) - g0, gl);
            }
            const float av = fmaf(G0 + g0, dl, gl * ((1.f + d0) + dl));
            const float GA = G0 + (Aref + av);
            const float S = fmaf(sa, ua - u0[a], sb * (ub - u0[b]));
            const float tau = av - GA * lk * h * S;
            f[a] = fmaf(sa * (h / 15.f), tau, f[a]);
            f[b] = fmaf(sb * (h / 15.f), tau, f[b]);
            if (cc) *cc += (1.f / 15.f) * (GA * h * S);
        }
        return;
    }
    // planes (x, z), (y, z): the + and - members (in-plane sign) of each z
    // side, their in-plane difference from corner differences
    float da = 0.f, db = 0.f;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const float sb = side ? -1.f : 1.f;
        const int m = 2 * side, mp = 2 * side + 1;  // in-plane sign +, -
        float dm = 0.f, dpp = 0.f, Dd = 0.f, gm = 0.f, gp = 0.f, Dg = 0.f;
        float am = 0.f, ap = 0.f, bm = 0.f, bp = 0.f, Db = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float w = P.sh.nb_w[PL][k], wm = P.sh.md_w[PL][k];
            const float n1 = __ldg(fl.dn + nb(m, k)), n2 = __ldg(fl.dn + nb(mp, k));
            const float b1 = __ldg(fb + nb(m, k)), b2 = __ldg(fb + nb(mp, k));
            const float g1 = __ldg(fl.dG + md(m, k)), g2 = __ldg(fl.dG + md(mp, k));
            dm = fmaf(w, n1, dm);
            dpp = fmaf(w, n2, dpp);
            Dd = fmaf(w, n1 - n2, Dd);
            bm = fmaf(w, b1, bm);
            bp = fmaf(w, b2, bp);
            Db = fmaf(w, b1 - b2, Db);
            gm = fmaf(wm, g1, gm);
            gp = fmaf(wm, g2, gp);
            Dg = fmaf(wm, g1 - g2, Dg);
            am = fmaf(w, __ldg(fa + nb(m, k)), am);
            ap = fmaf(w, __ldg(fa + nb(mp, k)), ap);
        }
        const float Am = shell_A(dm, gm, G0), Ap = shell_A(dpp, gp, G0);
        const float DA = fmaf(G0, Dd, fmaf(Dg, 1.f + dm, gp * Dd));
        const float c1 = (G0 + Am) * lk * h, c2 = (G0 + Ap) * lk * h, Dc = DA * lk * h;
        const float xm = am - u0[a], xp = ap - u0[a], zm = bm - u0[b], zp = bp - u0[b];
        da += DA - fmaf(c1, xm, c2 * xp) - sb * fmaf(c1, Db, Dc * zp);
        db += sb * ((Am + Ap) - fmaf(c1, xm, -c2 * xp) - sb * fmaf(c1, zm, c2 * zp));
        if (cc) *cc += (1.f / 15.f) * h * ((G0 + Am) * (xm + sb * zm) + (G0 + Ap) * (-xp + sb * zp));
    }
    f[a] += (h / 15.f) * da;
    f[b] += (h / 15.f) * db;
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

// Paired FP32 arithmetic on nodes (j, j + 1) of a v4: one instruction does
// both nodes (fma / add / mul .f32x2, sm_100 and later); each component
// rounds as the scalar operation does.
__device__ __forceinline__ float2 p2(const v4 r, int j) { return make_float2(r[j], r[j + 1]); }
__device__ __forceinline__ void put2(v4 r, int j, float2 v)
{
    r[j] = v.x;
    r[j + 1] = v.y;
}
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
// a - b, rounded once (b (-1) is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bc2(-1.f), a); }
// shell_A of a pair: G0 dq + gq (1 + dq)
__device__ __forceinline__ float2 shell_A2(float2 dq, float2 gq, float G0)
{
    return fma2(bc2(G0), dq, mul2(gq, add2(bc2(1.f), dq)));
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

// Mirror images along x (and y) of the shell points carry the x (y) force as
// a small difference of large values next to a wall (density layering, wall-
// normal velocity u_z ~ 0.1), so those differences are formed before any
// large value is rounded: the points of the (x, y) plane are interpolated
// relative to the node's own n and g2 values (all members then are small
// in-plane deviations), the pairs of the (x, z) and (y, z) planes that share
// the z offset as corner-by-corner differences, and the x and y axis pairs as
// differences of the loaded values. With A = G0 dq + gq (1 + dq):
//   A - A' = G0 (dq - dq') + (gq - gq') (1 + dq) + gq' (dq - dq').

// interpolants of member M of plane PL (0: (x, y), 1: (x, z); a = x) from
// its x-window corners; REF: n and g2 relative to the node's own values
template <int SIG, int PL, int M, bool LN, bool REF>
__device__ __forceinline__ void member_x(const Params& P, const Fields& fl, int pb, const v4 d0, const v4 g0, v4 dq,
                                         v4 ua, v4 ub, v4 gq, Lanes ln)
{
    constexpr int LO = cisqrt(SIG * SIG / 2), LOM = cisqrt((SIG / 2) * (SIG / 2) / 2);
    constexpr int SA = (M & 1) ? -1 : 1, SB = (M & 2) ? -1 : 1;
    const int sbs = PL == 0 ? P.g.px : P.g.px * P.g.py;
    const float* fb = PL == 0 ? fl.uy : fl.uz;
#pragma unroll
    for (int kb = 0; kb < 2; ++kb) {
        const int row = pb + SB * (LO + kb) * sbs;
        const float w0 = P.sh.nb_w[PL][2 * kb], w1 = P.sh.nb_w[PL][2 * kb + 1];
        v4 c0, c1;
        // acc += w0 (c0 - r) + w1 (c1 - r), r the reference (REF) or 0
        auto interp = [&](float a0, float a1, const v4 r, v4 acc) {
#pragma unroll
            for (int j = 0; j < 4; j += 2) {
                float2 e0 = p2(c0, j), e1 = p2(c1, j);
                if (REF && r) {
                    e0 = sub2(e0, p2(r, j));
                    e1 = sub2(e1, p2(r, j));
                }
                put2(acc, j, fma2(bc2(a1), e1, fma2(bc2(a0), e0, p2(acc, j))));
            }
        };
        corners_x<LO, SA, LN>(fl.dn, row, c0, c1, ln);
        interp(w0, w1, d0, dq);
        corners_x<LO, SA, LN>(fl.ux, row, c0, c1, ln);
        interp(w0, w1, nullptr, ua);
        corners_x<LO, SA, LN>(fb, row, c0, c1, ln);
        interp(w0, w1, nullptr, ub);
        const int mrow = pb + SB * (LOM + kb) * sbs;
        const float v0 = P.sh.md_w[PL][2 * kb], v1 = P.sh.md_w[PL][2 * kb + 1];
        corners_x<LOM, SA, LN>(fl.dG, mrow, c0, c1, ln);
        interp(v0, v1, g0, gq);
    }
}

// plane (x, y): the four members relative to the node's own n and g2 (d0,
// g0); their terms tau = T - T_ref share one reference, so both force
// components are sums of small accurate values
template <int SIG, bool C2, bool LN>
__device__ __forceinline__ void quartet_xy(const Params& P, const Fields& fl, int pb, const v4 d0, const v4 g0,
                                           const v4 u0[3], float G0, float lk, v4 f[3], v4 cc, Lanes ln)
{
    constexpr float h = 0.70710678118654752f, c = h / 15.f;
    auto one = [&](auto mc) {
        constexpr int M = decltype(mc)::value;
        constexpr float sa = (M & 1) ? -1.f : 1.f, sb = (M & 2) ? -1.f : 1.f;
        v4 dl, ua, ub, gl;
#pragma unroll
        for (int j = 0; j < 4; ++j) dl[j] = ua[j] = ub[j] = gl[j] = 0.f;
        member_x<SIG, 0, M, LN, true>(P, fl, pb, d0, g0, dl, ua, ub, gl, ln);
#pragma unroll
        for (int j = 0; j < 4; j += 2) {
            const float2 d = p2(d0, j), gg = p2(g0, j), dlj = p2(dl, j), opd = add2(bc2(1.f), d);
            const float2 Aref = fma2(bc2(G0), d, mul2(gg, opd));
            const float2 a = fma2(add2(bc2(G0), gg), dlj, mul2(p2(gl, j), add2(opd, dlj)));
            const float2 GA = add2(bc2(G0), add2(Aref, a));
            const float2 S = fma2(bc2(sa), sub2(p2(ua, j), p2(u0[0], j)), mul2(bc2(sb), sub2(p2(ub, j), p2(u0[1], j))));
            const float2 tau = fma2(mul2(GA, bc2(-lk * h)), S, a);
            put2(f[0], j, fma2(bc2(sa * c), tau, p2(f[0], j)));
            put2(f[1], j, fma2(bc2(sb * c), tau, p2(f[1], j)));
            if constexpr (C2) put2(cc, j, fma2(bc2(h / 15.f), mul2(GA, S), p2(cc, j)));
        }
    };
    one(std::integral_constant<int, 0>{});
    one(std::integral_constant<int, 1>{});
    one(std::integral_constant<int, 2>{});
    one(std::integral_constant<int, 3>{});
}

// plane (x, z) (PL 1) or (y, z) (PL 2): the two members with z offset sign SB
// and opposite in-plane sign: their interpolants d, g, ua, ub (m: +, p: -)
// and the corner-by-corner differences of d, g and ub
template <int SIG, int PL, int SB, bool LN>
__device__ __forceinline__ void pair_interp(const Params& P, const Fields& fl, int pb, v4 dm, v4 dp, v4 Dd, v4 gm,
                                            v4 gp, v4 Dg, v4 am, v4 ap, v4 bm, v4 bp, v4 Db, Lanes ln)
{
    constexpr int LO = cisqrt(SIG * SIG / 2), LOM = cisqrt((SIG / 2) * (SIG / 2) / 2);
    const float* fa = PL == 1 ? fl.ux : fl.uy;
    const int sz = P.g.px * P.g.py;
    // corner values of the + and - members of one field (accumulated with weight w)
    auto acc = [&](const float* f, const v4 cp, const v4 cm, float w, v4 im, v4 ip, v4 D) {
#pragma unroll
        for (int j = 0; j < 4; j += 2) {
            const float2 a = p2(cp, j), b = p2(cm, j), W = bc2(w);
            put2(im, j, fma2(W, a, p2(im, j)));
            put2(ip, j, fma2(W, b, p2(ip, j)));
            if (D) put2(D, j, fma2(W, sub2(a, b), p2(D, j)));
        }
    };
    if constexpr (PL == 1) {
#pragma unroll
        for (int kb = 0; kb < 2; ++kb) {
            const int row = pb + SB * (LO + kb) * sz;
            const float w0 = P.sh.nb_w[1][2 * kb], w1 = P.sh.nb_w[1][2 * kb + 1];
            v4 c0, c1, e0, e1;
            corners_x<LO, 1, LN>(fl.dn, row, c0, c1, ln);
            corners_x<LO, -1, LN>(fl.dn, row, e0, e1, ln);
            acc(fl.dn, c0, e0, w0, dm, dp, Dd);
            acc(fl.dn, c1, e1, w1, dm, dp, Dd);
            corners_x<LO, 1, LN>(fa, row, c0, c1, ln);
            corners_x<LO, -1, LN>(fa, row, e0, e1, ln);
            acc(fa, c0, e0, w0, am, ap, nullptr);
            acc(fa, c1, e1, w1, am, ap, nullptr);
            corners_x<LO, 1, LN>(fl.uz, row, c0, c1, ln);
            corners_x<LO, -1, LN>(fl.uz, row, e0, e1, ln);
            acc(fl.uz, c0, e0, w0, bm, bp, Db);
            acc(fl.uz, c1, e1, w1, bm, bp, Db);
            const int mrow = pb + SB * (LOM + kb) * sz;
            const float v0 = P.sh.md_w[1][2 * kb], v1 = P.sh.md_w[1][2 * kb + 1];
            corners_x<LOM, 1, LN>(fl.dG, mrow, c0, c1, ln);
            corners_x<LOM, -1, LN>(fl.dG, mrow, e0, e1, ln);
            acc(fl.dG, c0, e0, v0, gm, gp, Dg);
            acc(fl.dG, c1, e1, v1, gm, gp, Dg);
        }
    } else {
        const int sy = P.g.px;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int ka = k & 1, kb = k >> 1;
            const int o = pb + (LO + ka) * sy + SB * (LO + kb) * sz;
            const int om = pb - (LO + ka) * sy + SB * (LO + kb) * sz;
            const int q = pb + (LOM + ka) * sy + SB * (LOM + kb) * sz;
            const int qm = pb - (LOM + ka) * sy + SB * (LOM + kb) * sz;
            const float w = P.sh.nb_w[2][k], wm = P.sh.md_w[2][k];
            v4 c, e;
            set4(c, ld4(fl.dn + o));
            set4(e, ld4(fl.dn + om));
            acc(fl.dn, c, e, w, dm, dp, Dd);
            set4(c, ld4(fa + o));
            set4(e, ld4(fa + om));
            acc(fa, c, e, w, am, ap, nullptr);
            set4(c, ld4(fl.uz + o));
            set4(e, ld4(fl.uz + om));
            acc(fl.uz, c, e, w, bm, bp, Db);
            set4(c, ld4(fl.dG + q));
            set4(e, ld4(fl.dG + qm));
            acc(fl.dG, c, e, wm, gm, gp, Dg);
        }
    }
}

// one z side (sign SB) of plane (x, z) or (y, z): T_+ - T_- (the in-plane
// force) from the differences, SB (T_+ + T_-) (the z force) directly
template <int SIG, int PL, int SB, bool C2, bool LN>
__device__ __forceinline__ void pair_terms(const Params& P, const Fields& fl, int pb, const v4 u0[3], float G0,
                                           float lk, v4 da, v4 db, v4 cc, Lanes ln)
{
    constexpr int a = PL == 1 ? 0 : 1;
    constexpr float h = 0.70710678118654752f, sb = (float)SB;
    v4 dm, dp, Dd, gm, gp, Dg, am, ap, bm, bp, Db;
#pragma unroll
    for (int j = 0; j < 4; ++j) dm[j] = dp[j] = Dd[j] = gm[j] = gp[j] = Dg[j] = am[j] = ap[j] = bm[j] = bp[j] = Db[j] = 0.f;
    pair_interp<SIG, PL, SB, LN>(P, fl, pb, dm, dp, Dd, gm, gp, Dg, am, ap, bm, bp, Db, ln);
    const float2 one = bc2(1.f), g0 = bc2(G0), lkh = bc2(lk * h), SB2 = bc2(sb);
#pragma unroll
    for (int j = 0; j < 4; j += 2) {
        const float2 dmj = p2(dm, j), dpj = p2(dp, j), Ddj = p2(Dd, j);
        const float2 Am = shell_A2(dmj, p2(gm, j), G0), Ap = shell_A2(dpj, p2(gp, j), G0);
        const float2 DA = fma2(g0, Ddj, fma2(p2(Dg, j), add2(one, dmj), mul2(p2(gp, j), Ddj)));
        const float2 Gm = add2(g0, Am), Gp = add2(g0, Ap);
        const float2 cm = mul2(Gm, lkh), cp = mul2(Gp, lkh), Dc = mul2(DA, lkh);
        const float2 xm = sub2(p2(am, j), p2(u0[a], j)), xp = sub2(p2(ap, j), p2(u0[a], j));  // in-plane offsets
        const float2 zm = sub2(p2(bm, j), p2(u0[2], j)), zp = sub2(p2(bp, j), p2(u0[2], j));  // wall-normal offsets
        // T = A - c (s_a (u_a - u0_a) + s_b (u_z - u0_z)), s_a = +1 for m, -1 for p
        const float2 ta = sub2(sub2(DA, fma2(cm, xm, mul2(cp, xp))), mul2(SB2, fma2(cm, p2(Db, j), mul2(Dc, zp))));
        put2(da, j, add2(p2(da, j), ta));
        const float2 tb = sub2(sub2(add2(Am, Ap), sub2(mul2(cm, xm), mul2(cp, xp))),
                               mul2(SB2, fma2(cm, zm, mul2(cp, zp))));
        put2(db, j, fma2(SB2, tb, p2(db, j)));
        if constexpr (C2)
            put2(cc, j, fma2(bc2(h / 15.f), fma2(Gm, fma2(SB2, zm, xm), mul2(Gp, fma2(SB2, zp, mul2(bc2(-1.f), xp)))),
                             p2(cc, j)));
    }
}

template <int SIG, int PL, bool C2, bool LN>
__device__ __forceinline__ void quartet_z(const Params& P, const Fields& fl, int pb, const v4 u0[3], float G0,
                                          float lk, v4 f[3], v4 cc, Lanes ln)
{
    constexpr int a = PL == 1 ? 0 : 1;
    constexpr float c = 0.70710678118654752f / 15.f;
    v4 da, db;
#pragma unroll
    for (int j = 0; j < 4; ++j) da[j] = db[j] = 0.f;
    pair_terms<SIG, PL, 1, C2, LN>(P, fl, pb, u0, G0, lk, da, db, cc, ln);
    pair_terms<SIG, PL, -1, C2, LN>(P, fl, pb, u0, G0, lk, da, db, cc, ln);
#pragma unroll
    for (int j = 0; j < 4; j += 2) {
        put2(f[a], j, fma2(bc2(c), p2(da, j), p2(f[a], j)));
        put2(f[2], j, fma2(bc2(c), p2(db, j), p2(f[2], j)));
    }
}

template <int SIG, int A, bool C2>
__device__ __forceinline__ void axis4(const Params& P, const Fields& fl, int pb, const v4 u0[3], float G0, float lk,
                                      v4 f[3], v4 cc)
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
    for (int j = 0; j < 4; j += 2) {
        const float2 dpj = p2(dp, j), dmj = p2(dm, j), gpj = p2(gp, j), gmj = p2(gm, j), u0j = p2(u0[A], j);
        const float2 Ap = shell_A2(dpj, gpj, G0), Am = shell_A2(dmj, gmj, G0);
        // A_+ - A_-: from the differences of the loaded values along x and y
        float2 DA;
        if constexpr (A == 2) {
            DA = sub2(Ap, Am);
        } else {
            const float2 dd = sub2(dpj, dmj);
            DA = fma2(bc2(G0), dd, fma2(sub2(gpj, gmj), add2(bc2(1.f), dpj), mul2(gmj, dd)));
        }
        const float2 wp = mul2(add2(bc2(G0), Ap), sub2(p2(up, j), u0j));
        const float2 wm = mul2(add2(bc2(G0), Am), sub2(u0j, p2(um, j)));
        put2(f[A], j, fma2(bc2(1.f / 30.f), fma2(bc2(-lk), sub2(wp, wm), DA), p2(f[A], j)));
        if constexpr (C2) put2(cc, j, fma2(bc2(1.f / 30.f), add2(wp, wm), p2(cc, j)));
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
#ifndef FORCE_MINB
#define FORCE_MINB (512 / FORCE_NT)
#endif
template <int SIG, bool C2, bool LN>
__global__ void __launch_bounds__(FORCE_NT, FORCE_MINB) k_force4(Params P, TileMap tm, Fields fl,
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
    v4 d0, g0, u0[3];
    set4(d0, ld4(fl.dn + pb));
    set4(g0, ld4(fl.dG + pb));
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
        quartet_xy<SIG, C2, LN>(P, fl, pb, d0, g0, u0, S.G0, lk, f, cc, ln);
        quartet_z<SIG, 1, C2, LN>(P, fl, pb, u0, S.G0, lk, f, cc, ln);
        quartet_z<SIG, 2, C2, LN>(P, fl, pb, u0, S.G0, lk, f, cc, ln);
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
// steps 5-6 with step 1 of the next step, in pull form (Sec. Methods: the
// forward-Euler update with the first-order source towards the local
// equilibrium; half-way bounce-back at the walls). Every node gathers the
// populations that stream into it, applies to each the collision of its
// source node, and forms the new moments from the 19 values it holds, so the
// populations are read and written once per step.
//
// Stored populations. A node's populations are kept as
//   h_i = s_T (f_i - f_i^eq(n, u)) / (w_i n),
// the non-equilibrium part of f_i relative to the node's equilibrium weight
// w_i n, at the moments n, u of the step they belong to (the field buffers of
// that step hold those moments in FP32); s_T = 2^8 with FP16 storage (keeps
// the small parts of the bulk clear of the FP16 subnormal range) and 1 with
// FP32. The equilibrium part, which carries the flow, is never rounded to the
// storage type. In units of w_i n0, with dn = n/n0 - 1 and
// e_i = (1 + dn)(3 c.u + 9/2 (c.u)^2 - 3/2 u.u),
//   f_i / (w_i n0) - 1 = dn + e_i + (1 + dn) h_i / s_T.
// BGK towards f^eq(n, u) with omega = 1/tau, plus the source
// 3 c.F + (3/2) F.w (|c|^2 - 1) (F the force per n0, F.w the energy source
// when on), gives the post-collision value
//   f_i' / (w_i n0) - 1 = dn + T_i + m h_i,  m = (1 - omega)(1 + dn) / s_T,
//   T_i = e_i + 3 c.F + (3/2) F.w (|c|^2 - 1),
// and T splits by lattice-velocity class into
//   axis a, sign s:            s P_a + C_a
//   plane (a, b), signs sa sb: sa P_a + sb P_b + C_ab + sa sb X_ab
//   rest:                      C_0
// with q = 1 + dn, P = 3 (q u + F), B = -(3/2) q u.u, C_a = B + (9/2) q u_a^2,
// C_ab = B + (9/2) q (u_a^2 + u_b^2) + (3/2) F.w, X_ab = 9 q u_a u_b and
// C_0 = B - (3/2) F.w = (2 (C_x + C_y + C_z) - (C_xy + C_xz + C_yz)) / 3.
// The value reaching r from s = r - c_i, relative to dn(r), is
// v_i = T_i(s) + m(s) h_i(s) + (dn(s) - dn(r)); at a wall it is the node's own
// post-collision value of the opposite direction (c -> -c: the P terms change
// sign). The new moments are dn(r) + S, S = sum_i w_i v_i, and
// u = sum_i w_i c_i v_i / (1 + dn(r) + S); the new populations are stored as
// their non-equilibrium parts at those moments.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ constexpr float store_scale() { return sizeof(T) == 2 ? 256.f : 1.f; }

// staged quantities of a node: dn, P_x..z, C_x..z, C_xy C_xz C_yz, X_xy X_xz X_yz
constexpr int SQ_DN = 0, SQ_P = 1, SQ_CA = 4, SQ_CP = 7, SQ_X = 10, CSM_NF = 13;

// The staged quantities of a node from its moments and force; st(k, value)
// receives quantity k. Each quantity ends in a rounding intrinsic (never
// merged into a later multiply-add), so a kernel that uses them at once and
// one that stores them first compute identical values.
//
// shifted (velocity-shifted second-order forcing, the force F from the
// unshifted moments): BGK towards f^eq(n, u') with u' = u + F/(2 q), and the
// source k [3 (c - u').F + 9 (c.u')(c.F)], k = 1 - omega/2. T_i is then
// (1 - omega) e_i(u) + omega e_i(u') + that source, whose class split, with
// T = alpha + beta.c + c.gamma.c, is P_a = beta_a, C_a = alpha + gamma_aa,
// C_ab = alpha + gamma_aa + gamma_bb, X_ab = 2 gamma_ab:
//   alpha   = -(3/2) q ((1 - omega) u.u + omega u'.u') - 3 k u'.F
//   beta_a  = 3 q ((1 - omega) u_a + omega u'_a) + 3 k F_a
//   gamma_ab = (9/2) q ((1 - omega) u_a u_b + omega u'_a u'_b) + (9/2) k (u'_a F_b + u'_b F_a).
template <class St>
__device__ __forceinline__ void src_terms(float d, float ux, float uy, float uz, float4 f, float om, bool shifted,
                                          St st)
{
    const float q1 = 1.f + d;
    st(SQ_DN, d);
    if (shifted) {
        const float hq = 0.5f / q1;
        const float vx = fmaf(hq, f.x, ux), vy = fmaf(hq, f.y, uy), vz = fmaf(hq, f.z, uz);  // u'
        const float k = fmaf(-0.5f, om, 1.f), a1 = 1.f - om;
        const float uu = ux * ux + uy * uy + uz * uz, vv = vx * vx + vy * vy + vz * vz;
        const float vF = vx * f.x + vy * f.y + vz * f.z;
        const float alpha = fmaf(-1.5f * q1, fmaf(a1, uu, om * vv), -3.f * k * vF);
        const float u[3] = {ux, uy, uz}, v[3] = {vx, vy, vz}, F[3] = {f.x, f.y, f.z};
        auto gam = [&](int a, int b) {
            return fmaf(4.5f * q1, fmaf(a1, u[a] * u[b], om * (v[a] * v[b])), 4.5f * k * fmaf(v[a], F[b], v[b] * F[a]));
        };
        const float gxx = gam(0, 0), gyy = gam(1, 1), gzz = gam(2, 2);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            st(SQ_P + a, __fmul_rn(3.f, fmaf(q1, fmaf(a1, u[a], om * v[a]), k * F[a])));
        st(SQ_CA + 0, __fadd_rn(alpha, gxx));
        st(SQ_CA + 1, __fadd_rn(alpha, gyy));
        st(SQ_CA + 2, __fadd_rn(alpha, gzz));
        st(SQ_CP + 0, __fadd_rn(alpha, gxx + gyy));
        st(SQ_CP + 1, __fadd_rn(alpha, gxx + gzz));
        st(SQ_CP + 2, __fadd_rn(alpha, gyy + gzz));
        st(SQ_X + 0, __fmul_rn(2.f, gam(0, 1)));
        st(SQ_X + 1, __fmul_rn(2.f, gam(0, 2)));
        st(SQ_X + 2, __fmul_rn(2.f, gam(1, 2)));
        return;
    }
    const float B = __fmul_rn(-1.5f * q1, ux * ux + uy * uy + uz * uz);
    const float a = 4.5f * q1, ax = a * ux * ux, ay = a * uy * uy, az = a * uz * uz;
    const float fw = 1.5f * f.w, b = 9.f * q1;
    st(SQ_P + 0, __fmul_rn(3.f, fmaf(q1, ux, f.x)));
    st(SQ_P + 1, __fmul_rn(3.f, fmaf(q1, uy, f.y)));
    st(SQ_P + 2, __fmul_rn(3.f, fmaf(q1, uz, f.z)));
    st(SQ_CA + 0, __fadd_rn(B, ax));
    st(SQ_CA + 1, __fadd_rn(B, ay));
    st(SQ_CA + 2, __fadd_rn(B, az));
    st(SQ_CP + 0, __fadd_rn(B + (ax + ay), fw));
    st(SQ_CP + 1, __fadd_rn(B + (ax + az), fw));
    st(SQ_CP + 2, __fadd_rn(B + (ay + az), fw));
    st(SQ_X + 0, __fmul_rn(b * ux, uy));
    st(SQ_X + 1, __fmul_rn(b * ux, uz));
    st(SQ_X + 2, __fmul_rn(b * uy, uz));
}

// v_i (see above) from the source's staged quantities sl (quantity k at
// sl[k * ST]) and its stored h; wall: sl is the node itself and the
// direction arrives reversed
template <int i, int ST>
__device__ __forceinline__ float arrive(const float* sl, float h, float om1s, float dnr, bool wall)
{
    constexpr int cx = kCx(i), cy = kCy(i), cz = kCz(i);
    const float sg = wall ? -1.f : 1.f;
    float t;
    if constexpr (i == 0) {
        t = (2.f * (sl[(SQ_CA + 0) * ST] + sl[(SQ_CA + 1) * ST] + sl[(SQ_CA + 2) * ST]) -
             (sl[(SQ_CP + 0) * ST] + sl[(SQ_CP + 1) * ST] + sl[(SQ_CP + 2) * ST])) *
            (1.f / 3.f);
    } else if constexpr (kC2(i) == 1) {
        constexpr int a = cx ? 0 : (cy ? 1 : 2);
        constexpr float ca = (float)(cx + cy + cz);
        t = fmaf(sg * ca, sl[(SQ_P + a) * ST], sl[(SQ_CA + a) * ST]);
    } else {
        constexpr int pl = cz == 0 ? 0 : (cy == 0 ? 1 : 2);
        constexpr int a = pl == 2 ? 1 : 0, b = pl == 0 ? 1 : 2;
        constexpr float ca = (float)(a == 0 ? cx : cy), cb = (float)(b == 1 ? cy : cz);
        t = sl[(SQ_CP + pl) * ST] + sg * (ca * sl[(SQ_P + a) * ST] + cb * sl[(SQ_P + b) * ST]) +
            (ca * cb) * sl[(SQ_X + pl) * ST];
    }
    const float ds = sl[SQ_DN * ST];
    return fmaf(fmaf(om1s, ds, om1s), h, t) + (ds - dnr);
}

// fn(std::integral_constant<int, i>) for i = 0 .. Q-1, unrolled at compile time
template <class Fn, int... I>
__device__ __forceinline__ void for_dirs_seq(Fn&& fn, std::integer_sequence<int, I...>)
{
    (fn(std::integral_constant<int, I>{}), ...);
}
template <class Fn>
__device__ __forceinline__ void for_dirs(Fn&& fn)
{
    for_dirs_seq(fn, std::make_integer_sequence<int, Q>{});
}

// Mirror pairs. The flow along x and y is a small signal next to the
// wall-normal velocity and force (u_z and F_z of O(0.1) where u_x ~ 1e-4), so
// the arriving values of directions that differ only in the sign of c_x (or
// c_y) share large parts. Their difference is therefore formed from the
// differences of the staged quantities of their two sources (which lie in
// the same plane, two nodes apart), and the x and y momenta are sums of those
// differences: a sum of separately rounded values of O(1) would carry the
// signal only to ~1e-7 of those values. Ten pairs (plus member first):
//   along x: (1,2) (7,10) (9,8) (11,14) (13,12); along y: (3,4) (7,9) (10,8) (15,18) (17,16).
// Directions 1 3 7 9 10 11 13 15 17 are derived: slot i holds v_i - v_b of
// its pair partner b (7 from 10, 10 from 8), the others ("base") hold v_i.
template <int i, int ip>
struct Mirror {
    static constexpr int A = kCx(i) != kCx(ip) ? 0 : 1;  // the component that changes sign
    static constexpr bool axis = kC2(i) == 1;
    // the shared nonzero component of a plane direction and its sign
    static constexpr int B = axis ? 0 : (A == 0 ? (kCy(i) != 0 ? 1 : 2) : (kCx(i) != 0 ? 0 : 2));
    static constexpr int PL = (A == 2 || B == 2) ? (A == 0 || B == 0 ? 1 : 2) : 0;
    static constexpr float CB = axis ? 0.f : (float)(B == 0 ? kCx(i) : (B == 1 ? kCy(i) : kCz(i)));
};

// v_i - v_ip of a mirror pair (staged quantities of the sources at s and sp,
// stride ST; the stored values h, hp of the two directions; wall: both
// arrive reversed from the node itself, s = sp)
template <int i, int ip, int ST>
__device__ __forceinline__ float mirror_diff(const float* s, const float* sp, float h, float hp, float om1s, bool wall)
{
    using M = Mirror<i, ip>;
    const float sg = wall ? -1.f : 1.f;
    float dt;
    if constexpr (M::axis) {
        dt = (s[(SQ_CA + M::A) * ST] - sp[(SQ_CA + M::A) * ST]) + sg * (s[(SQ_P + M::A) * ST] + sp[(SQ_P + M::A) * ST]);
    } else {
        dt = (s[(SQ_CP + M::PL) * ST] - sp[(SQ_CP + M::PL) * ST]) +
             sg * (s[(SQ_P + M::A) * ST] + sp[(SQ_P + M::A) * ST]) +
             (sg * M::CB) * (s[(SQ_P + M::B) * ST] - sp[(SQ_P + M::B) * ST]) +
             M::CB * (s[(SQ_X + M::PL) * ST] + sp[(SQ_X + M::PL) * ST]);
    }
    const float ds = s[SQ_DN * ST], dsp = sp[SQ_DN * ST];
    // m(s) h - m(sp) hp with m = om1s (1 + d)
    const float dm = om1s * fmaf(1.f + ds, h - hp, (ds - dsp) * hp);
    return (dt + dm) + (ds - dsp);
}

// element off of direction i's part of a population buffer
template <typename T>
__device__ __forceinline__ T* pop_at(T* p, const Params& P, int i, long long off)
{
    return p + (P.dbase[i] + off);
}
// the same in place, where every element offset fits 32 bits: one 32-bit add
// and one widening multiply-add per address
template <typename T>
__device__ __forceinline__ T* pop_at_ip(T* p, const Params& P, int i, int slot)
{
    return p + (P.dbase32[i] + (unsigned)slot);
}

// the new moments of a node from its arriving values (slots as above, d79 =
// v_7 - v_9), then its populations stored as non-equilibrium parts at those
// moments (at(i): where direction i goes): base directions directly, derived
// ones as their partner's stored value plus the difference (so the pairs'
// differences survive the rounding of the large common parts); returns dn
// and writes u
template <typename T, class Addr>
__device__ __forceinline__ float pull_finish(Addr at, const float* v, float d79, float dnr, float& ux, float& uy,
                                             float& uz)
{
    constexpr float w1 = 1.f / 18.f, w2 = 1.f / 36.f;
    // arriving values of the derived directions
    const float v1 = v[2] + v[1], v3 = v[4] + v[3], v9 = v[8] + v[9], v10 = v[8] + v[10];
    const float v7 = v10 + v[7], v11 = v[14] + v[11], v13 = v[12] + v[13], v15 = v[18] + v[15];
    const float v17 = v[16] + v[17];
    const float S = (1.f / 3.f) * v[0] +
                    w1 * (((v1 + v[2]) + (v3 + v[4])) + (v[5] + v[6])) +
                    w2 * ((((v7 + v[8]) + (v9 + v10)) + ((v11 + v[12]) + (v13 + v[14]))) +
                          ((v15 + v[16]) + (v17 + v[18])));
    const float Jz = w1 * (v[5] - v[6]) +
                     w2 * (((v11 - v[12]) - (v13 - v[14])) + ((v15 - v[16]) - (v17 - v[18])));
    const float Jx = w1 * v[1] + w2 * (((v[7] + v[9]) + (v[11] + v[13])));
    const float Jy = w1 * v[3] + w2 * ((d79 + v[10]) + (v[15] + v[17]));
    const float dn = dnr + S;
    const float inv = 1.f / (1.f + dn);
    ux = Jx * inv;
    uy = Jy * inv;
    uz = Jz * inv;
    const float uu = ux * ux + uy * uy + uz * uz;
    constexpr float sT = store_scale<T>();
    auto p_of = [&](int i) {  // f_i^eq / (w_i n) - 1
        const float cu = dot_c(i, ux, uy, uz);
        return fmaf(cu, fmaf(4.5f, cu, 3.f), -1.5f * uu);
    };
    auto base = [&](int i, float vi) { return (vi - S) * inv - p_of(i); };
    // p_i - p_ip of a pair that differs in component a: u_a (6 + 18 R),
    // R = the shared part of c.u
    auto dp = [&](float ua, float R) { return ua * fmaf(18.f, R, 6.f); };
    auto put = [&](int i, float h) { stp(at(i), sT * h); };
    put(0, base(0, v[0]));
    put(5, base(5, v[5]));
    put(6, base(6, v[6]));
    const float h2 = base(2, v[2]), h4 = base(4, v[4]), h8 = base(8, v[8]);
    put(2, h2);
    put(1, h2 + (v[1] * inv - dp(ux, 0.f)));
    put(4, h4);
    put(3, h4 + (v[3] * inv - dp(uy, 0.f)));
    put(8, h8);
    put(9, h8 + (v[9] * inv - dp(ux, -uy)));
    const float h10 = h8 + (v[10] * inv - dp(uy, -ux));
    put(10, h10);
    put(7, h10 + (v[7] * inv - dp(ux, uy)));
    const float h12 = base(12, v[12]), h14 = base(14, v[14]);
    put(12, h12);
    put(13, h12 + (v[13] * inv - dp(ux, -uz)));
    put(14, h14);
    put(11, h14 + (v[11] * inv - dp(ux, uz)));
    const float h16 = base(16, v[16]), h18 = base(18, v[18]);
    put(16, h16);
    put(17, h16 + (v[17] * inv - dp(uy, -uz)));
    put(18, h18);
    put(15, h18 + (v[15] * inv - dp(uy, uz)));
    return dn;
}

// moments of a node written to the next step's fields (with their images)
__device__ __forceinline__ void put_fields(const Params& P, const CsmIO& io, int x, int y, int z, float dn, float ux,
                                           float uy, float uz, int* status)
{
    if (!(1.f + dn > 0.f) || !isfinite(dn) || !isfinite(ux + uy + uz)) atomicOr(status, 1);
    auto put = [&](int p) {
        io.dnw[p] = dn;
        io.uxw[p] = ux;
        io.uyw[p] = uy;
        io.uzw[p] = uz;
    };
    if (no_images(P.g, x, y, z))
        put(pidx(P.g, x, y, z));
    else
        for_images(P.g, x, y, z, put);
}

// What a source node contributes is staged per node in shared memory: a CTA
// owns a 32 x 4 tile of x-y nodes, keeps three planes of it (plus a one-node
// halo) in a ring, and marches up a segment of z planes.
// 32 x 4 tiles of 128 threads, six CTAs per SM (measured at 512 x 512 x 192, sigma 12, same
// state: 32 x 4 / 128 threads / 6 CTAs 2.186 ms, 32 x 8 / 256 / 3 2.334 ms, 32 x 12 / 384 / 2
// 2.508 ms): more, smaller CTAs keep more population loads in flight across the two barriers
// of each plane
constexpr int CSM_TX = 32, CSM_TY = 4, CSM_THREADS = CSM_TX * CSM_TY;
constexpr int CSM_HX = CSM_TX + 2, CSM_HN = CSM_HX * (CSM_TY + 2);  // staged nodes per plane
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
    const int pq = (q + g.hw) * g.py * g.px;
    const float4* Fq = F + (long long)zq * g.ny * g.nx;
    const float om = P.sl[sq].inv_tau;
    const bool shifted = P.shifted != 0;
#pragma unroll
    for (int k = 0; k < CSM_KS; ++k) {
        if (k * NT >= CSM_HN || st.p[k] < 0) continue;
        const int h = threadIdx.x + k * NT;
        const int p = pq + st.p[k];
        src_terms(__ldg(io.dn + p), __ldg(io.ux + p), __ldg(io.uy + p), __ldg(io.uz + p), __ldg(Fq + st.n[k]), om,
                  shifted, [&](int j, float val) { slot[j * CSM_HN + h] = val; });
    }
}

// CTAs per SM the register budget is sized for (5 / 6 / 7 at 96 / 80 / 72
// registers: 2.57 / 2.39 / 2.55 ms at 512 x 512 x 192, sigma 12, FP32), and
// z planes per CTA segment
#ifndef CSM_MINB
#define CSM_MINB 6
#endif
#ifndef CSM_LZ
#define CSM_LZ 16
#endif

// the stored populations of directions [I0, I1) that stream into node
// (x, y, z): v[i - I0]; bit i of bb marks a direction that arrives from a
// wall (bounce-back: the node's own opposite population). IP: in place
// (slots from q, see above).
template <int I0, int I1, bool IP, typename T, bool RAW = false>
__device__ __forceinline__ void csm_pull(const Params& P, const T* __restrict__ pin, long long idx, int x, int y,
                                         int z, int zlo, int zhi, float* v, unsigned& bb, const IpSlots& q)
{
    const Geom& g = P.g;
    if constexpr (IP) {
#pragma unroll
        for (int i = I0; i < I1; ++i) {
            const int sz = z - kCz(i);
            if (!g.zper && (sz < zlo || sz > zhi)) {
                bb |= 1u << i;
                v[i - I0] = ldq<RAW>(pop_at_ip(pin, P, opp_of(i), q.wall_slot(i)));
            } else {
                v[i - I0] = ldq<RAW>(pop_at_ip(pin, P, i, q.slot(i)));
            }
        }
        return;
    }
    if (x > 0 && x < g.nx - 1 && y > 0 && y < g.ny - 1 && z > zlo && z < zhi) {
#pragma unroll
        for (int i = I0; i < I1; ++i) v[i - I0] = ldq<RAW>(pin + (idx + P.doff[i]));
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
            v[i - I0] = ldq<RAW>(pin + (P.dbase[opp_of(i)] + idx));
            continue;
        }
        v[i - I0] = ldq<RAW>(pin + (P.dbase[i] + (((long long)sz * g.ny + sy) * g.nx + sx)));
    }
}

// The arriving values of a node in the slots described at Mirror: the ten
// mirror differences first (from the stored values as loaded), then the ten
// base directions. src(i) is the source quantities of direction i (stride
// ST); wall directions arrive reversed from the node itself (own).
template <int ST, bool WALLS, class Src>
__device__ __forceinline__ void pull_gather_impl(Src src, const float* own, float om1s, float dnr, unsigned bb,
                                                 float* v, float& d79)
{
    auto wall = [&](int i) { return WALLS && ((bb >> i) & 1u) != 0u; };
    auto diff = [&](auto ic, auto ipc) {
        constexpr int i = decltype(ic)::value, ip = decltype(ipc)::value;
        const bool w = wall(i);
        return mirror_diff<i, ip, ST>(w ? own : src(ic), w ? own : src(ipc), v[i], v[ip], om1s, w);
    };
    using std::integral_constant;
    const float d7_10 = diff(integral_constant<int, 7>{}, integral_constant<int, 10>{});
    const float d9_8 = diff(integral_constant<int, 9>{}, integral_constant<int, 8>{});
    const float d10_8 = diff(integral_constant<int, 10>{}, integral_constant<int, 8>{});
    d79 = diff(integral_constant<int, 7>{}, integral_constant<int, 9>{});
    v[7] = d7_10;
    v[9] = d9_8;
    v[10] = d10_8;
    v[1] = diff(integral_constant<int, 1>{}, integral_constant<int, 2>{});
    v[3] = diff(integral_constant<int, 3>{}, integral_constant<int, 4>{});
    v[11] = diff(integral_constant<int, 11>{}, integral_constant<int, 14>{});
    v[13] = diff(integral_constant<int, 13>{}, integral_constant<int, 12>{});
    v[15] = diff(integral_constant<int, 15>{}, integral_constant<int, 18>{});
    v[17] = diff(integral_constant<int, 17>{}, integral_constant<int, 16>{});
    auto one = [&](auto ic) {
        constexpr int i = decltype(ic)::value;
        if constexpr (i == 0 || i == 2 || i == 4 || i == 5 || i == 6 || i == 8 || i == 12 || i == 14 || i == 16 ||
                      i == 18) {
            const bool w = i != 0 && wall(i);
            v[i] = arrive<i, ST>((i == 0 || w) ? own : src(ic), v[i], om1s, dnr, w);
        }
    };
    for_dirs(one);
}

// The arriving values of a node in the slots described at Mirror: the ten
// mirror differences first (from the stored values as loaded), then the ten
// base directions. src(i) is the source quantities of direction i (stride
// ST); wall directions arrive reversed from the node itself (own). Nodes
// with no wall direction (bb = 0, almost all) take a path without the wall
// selections.
template <int ST, class Src>
__device__ __forceinline__ void pull_gather(Src src, const float* own, float om1s, float dnr, unsigned bb, float* v,
                                            float& d79)
{
    if (bb == 0u)
        pull_gather_impl<ST, false>(src, own, om1s, dnr, bb, v, d79);
    else
        pull_gather_impl<ST, true>(src, own, om1s, dnr, bb, v, d79);
}

// the gather of a node staged at hc in the ring (planes below, own, above)
__device__ __forceinline__ void csm_collide(const float* own, const float* below, const float* above, int hc,
                                            float om1s, float dnr, unsigned bb, float* v, float& d79)
{
    auto src = [&](auto ic) -> const float* {
        constexpr int i = decltype(ic)::value;
        constexpr int cx = kCx(i), cy = kCy(i), cz = kCz(i);
        return (cz > 0 ? below : (cz < 0 ? above : own)) + hc - cx - cy * CSM_HX;
    };
    pull_gather<CSM_HN>(src, own + hc, om1s, dnr, bb, v, d79);
}

// one node per thread, a CTA per 32 x 4 tile and z segment (measured with the
// earlier storage: two threads per node, each gathering half of the
// directions and adding the partial moments through shared memory, ran
// slower at twice the warps). PF: the population gathers of the next plane
// are issued before the current plane is staged and collided, so they are in
// flight across both barriers (19 more live registers: five CTAs per SM).
// FP16 gathers stay raw until the collision (measured at 512 x 512 x 192,
// sigma 12: 2.71 -> 2.54 ms; on a 256-slit ensemble 0.388 -> 0.335 ms): the
// staging between the gathers and their use then hides their latency, as it
// does for FP32 values, which nothing touches before the collision
template <typename T>
constexpr bool F16_RAW = sizeof(T) == 2;
template <typename T, bool PF, bool IP>
__global__ void __launch_bounds__(CSM_THREADS, PF ? CSM_MINB - 1 : CSM_MINB)
    k_csm(Params P, const T* pin, T* pout, CsmIO io, const float4* __restrict__ F, int lz, int tiles_x, int tiles_y,
          int* status)
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
    // the population gathers of plane z (act: the node steps; om its 1/tau)
    // (in place, q returns the node's slots, which its stores reuse)
    auto gather = [&](int z, float* v, unsigned& bb, bool& act, float& om, IpSlots& q) {
        const int s = slit_of(P, z);
        act = in_xy && s >= 0 && !frozen(P, s);
        bb = 0;
        om = 0.f;
        if (act) {
            om = P.sl[s].inv_tau;
            if constexpr (IP) q = ip_slots(P, P.sl[s], s, x, y, z);
            csm_pull<0, Q, IP, T, F16_RAW<T>>(P, pin, ((long long)z * g.ny + y) * g.nx + x, x, y, z, P.sl[s].zlo,
                                              P.sl[s].zhi, v, bb, q);
        }
    };
    IpSlots qn, qz;
    float vn[Q];
    unsigned bbn = 0;
    bool actn = false;
    float omn = 0.f;
    if constexpr (PF) gather(zb, vn, bbn, actn, omn, qn);
    csm_stage<NT>(P, io, F, sm + csm_slot(zb - 1) * CSM_SLOT, st, zb - 1);
    csm_stage<NT>(P, io, F, sm + csm_slot(zb) * CSM_SLOT, st, zb);
    for (int z = zb; z < ze; ++z) {
        // issue the population loads first: they do not depend on the ring
        float v[Q];
        unsigned bb;
        bool act;
        float om;
        if constexpr (PF) {
#pragma unroll
            for (int i = 0; i < Q; ++i) v[i] = vn[i];
            bb = bbn;
            act = actn;
            om = omn;
            if (z + 1 < ze) gather(z + 1, vn, bbn, actn, omn, qn);
        } else {
            gather(z, v, bb, act, om, qz);
        }
        __syncthreads();  // the slot of plane z - 2 is free
        csm_stage<NT>(P, io, F, sm + csm_slot(z + 1) * CSM_SLOT, st, z + 1);
        __syncthreads();
        if (!act) continue;
        const long long idx = ((long long)z * g.ny + y) * g.nx + x;
        const float* own = sm + csm_slot(z) * CSM_SLOT;
        const float dnr = own[SQ_DN * CSM_HN + hc];
        float d79;
        if constexpr (F16_RAW<T>) {
#pragma unroll
            for (int k = 0; k < Q; ++k) v[k] = late_cvt(v[k]);
        }
        csm_collide(own, sm + csm_slot(z - 1) * CSM_SLOT, sm + csm_slot(z + 1) * CSM_SLOT, hc,
                    (1.f - om) / store_scale<T>(), dnr, bb, v, d79);
        float ux, uy, uz;
        float dn;
        if constexpr (IP) {
            // FP16: the stores reuse the gather's slots (2.64 -> 2.47 ms at
            // 512 x 512 x 192, sigma 12); FP32 recomputes them (holding them
            // across the collision spills there: 2.50 -> 2.57 ms)
            IpSlots q;
            if constexpr (PF || sizeof(T) == 4) {
                const int s = slit_of(P, z);
                q = ip_slots(P, P.sl[s], s, x, y, z);
            } else {
                q = qz;
            }
            dn = pull_finish<T>([&](int i) { return pop_at_ip(pout, P, i, q.slot(i)); }, v, d79, dnr, ux, uy, uz);
        } else {
            dn = pull_finish<T>([&](int i) { return pop_at(pout, P, i, idx); }, v, d79, dnr, ux, uy, uz);
        }
        put_fields(P, io, x, y, z, dn, ux, uy, uz, status);
    }
}

// The pull pass with its population gathers brought in by the tensor-memory
// accelerator (two-buffer layout). For every plane whose 19 sources lie
// inside the grid - interior tiles, no wall direction, away from the ends of
// a periodic z - one thread issues, one plane ahead, one copy per direction
// i of the tile's source box (the tile shifted by -c_i, widened in x to
// 16-byte boundaries: BW nodes from x0 - XM when c_ix = 1, else from x0;
// a 4-D tensor map: x, y, z, direction) into one of two shared-memory
// stages, completion counted in bytes on an mbarrier; the threads then read
// their 19 values from there. Other planes gather directly. The arithmetic
// is k_csm's (identical results).
template <typename T>
__host__ __device__ constexpr int tma_xm() { return sizeof(T) == 2 ? 8 : 4; }
template <typename T>
__host__ __device__ constexpr int tma_bw() { return CSM_TX + tma_xm<T>(); }
template <typename T>
__host__ __device__ constexpr int tma_box_bytes() { return tma_bw<T>() * CSM_TY * (int)sizeof(T); }
template <typename T>
__host__ __device__ constexpr int tma_box_pitch() { return (tma_box_bytes<T>() + 127) / 128 * 128; }
__host__ __device__ constexpr int csm_ring_bytes() { return (3 * CSM_SLOT * 4 + 127) / 128 * 128; }
template <typename T>
__host__ __device__ constexpr int csm_tma_smem_bytes() { return csm_ring_bytes() + 2 * Q * tma_box_pitch<T>() + 16; }

void pop_box(int storage, int* W, int* H)
{
    *W = storage == LBIF_STORE_F16 ? tma_bw<__half>() : tma_bw<float>();
    *H = CSM_TY;
}

template <typename T>
__global__ void __launch_bounds__(CSM_THREADS, 4)
    k_csm_tma(Params P, const __grid_constant__ CUtensorMap pmap, const T* pin, T* pout, CsmIO io,
              const float4* __restrict__ F, int lz, int tiles_x, int tiles_y, int* status)
{
    constexpr int NT = CSM_THREADS, XM = tma_xm<T>(), BW = tma_bw<T>(), BOX = tma_box_bytes<T>();
    constexpr int PB = tma_box_pitch<T>(), SB = Q * PB;
    extern __shared__ __align__(128) unsigned char smraw[];
    float* sm = reinterpret_cast<float*>(smraw);
    unsigned char* stg = smraw + csm_ring_bytes();
    uint64_t* mbar = reinterpret_cast<uint64_t*>(stg + 2 * SB);
    const Geom& g = P.g;
    const int tiles = tiles_x * tiles_y;
    const int tile = blockIdx.x % tiles, seg = blockIdx.x / tiles;
    const int x0 = (tile % tiles_x) * CSM_TX, y0 = (tile / tiles_x) * CSM_TY;
    const int t = threadIdx.x;
    const int tx = t % CSM_TX, ty = t / CSM_TX;
    const int x = x0 + tx, y = y0 + ty;
    const int hc = (ty + 1) * CSM_HX + tx + 1;
    const bool in_xy = x < g.nx && y < g.ny;
    const int zb = seg * lz, ze = min(zb + lz, g.nz);
    const bool interior = x0 >= 1 && x0 + CSM_TX <= g.nx - 1 && y0 >= 1 && y0 + CSM_TY <= g.ny - 1;
    // every source of plane z inside the grid and no wall direction (CTA-uniform)
    auto plane_tma = [&](int z) -> bool {
        if (!interior || z < 1 || z > g.nz - 2) return false;
        const int s = slit_of(P, z);
        if (s < 0 || frozen(P, s)) return false;
        return z > P.sl[s].zlo && z < P.sl[s].zhi;
    };
    if (t == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&pmap)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar + 1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int z) {  // one thread: the 19 boxes of plane z into stage z & 1
        const int b = z & 1;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar + b)),
                     "r"((uint32_t)(Q * BOX))
                     : "memory");
#pragma unroll
        for (int i = 0; i < Q; ++i)
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
                "%5}], [%6];" ::"r"(smem_addr(stg + b * SB + i * PB)),
                "l"(reinterpret_cast<uint64_t>(&pmap)), "r"(kCx(i) > 0 ? x0 - XM : x0), "r"(y0 - kCy(i)),
                "r"(z - kCz(i)), "r"(i), "r"(smem_addr(mbar + b))
                : "memory");
    };
    uint32_t pbits = 0u;  // bit b: the parity expected next on stage b
    uint32_t pend = 0u;  // bit b: stage b has copies in flight
    // bounded wait for stage b's copies; false if it ran out
    auto wait_stage = [&](int b) -> bool {
        long long spins = 0;
        bool ok;
        while (!(ok = mbar_wait_parity(mbar + b, (pbits >> b) & 1u)) && ++spins < BALL_WAIT_LIMIT) {
        }
        return ok;
    };
    const CsmStaged st = csm_staged<NT>(g, x0, y0);
    if (zb < ze && plane_tma(zb)) {
        if (t == 0) issue(zb);
        pend = 1u << (zb & 1);
    }
    csm_stage<NT>(P, io, F, sm + csm_slot(zb - 1) * CSM_SLOT, st, zb - 1);
    csm_stage<NT>(P, io, F, sm + csm_slot(zb) * CSM_SLOT, st, zb);
    for (int z = zb; z < ze; ++z) {
        const int s = slit_of(P, z);
        const bool act = in_xy && s >= 0 && !frozen(P, s);
        const bool tz = (pend >> (z & 1)) & 1u;
        float v[Q];
        unsigned bb = 0;
        const long long idx = ((long long)z * g.ny + y) * g.nx + x;
        const float om = act ? P.sl[s].inv_tau : 0.f;
        if (act && !tz) {
            IpSlots q;
            csm_pull<0, Q, false>(P, pin, idx, x, y, z, P.sl[s].zlo, P.sl[s].zhi, v, bb, q);
        }
        __syncthreads();  // ring slot of plane z - 2 and stage (z + 1) & 1 are free
        const bool tn = z + 1 < ze && plane_tma(z + 1);
        if (tn) {
            if (t == 0) issue(z + 1);
            pend |= 1u << ((z + 1) & 1);
        }
        csm_stage<NT>(P, io, F, sm + csm_slot(z + 1) * CSM_SLOT, st, z + 1);
        __syncthreads();
        if (tz) {
            const int b = z & 1;
            if (!__syncthreads_and(wait_stage(b))) {
                // record the timeout and wait (bounded) for the copies in flight
                if (t == 0) atomicOr(status, 4);
                if (tn) wait_stage((z + 1) & 1);
                return;
            }
            pbits ^= 1u << b;
            pend &= ~(1u << b);
            if (act) {
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const T* p = reinterpret_cast<const T*>(stg + b * SB + i * PB) + ty * BW +
                                 (tx - kCx(i) + (kCx(i) > 0 ? XM : 0));
                    if constexpr (sizeof(T) == 2)
                        v[i] = __half2float(*reinterpret_cast<const __half*>(p));
                    else
                        v[i] = *reinterpret_cast<const float*>(p);
                }
            }
        }
        if (!act) continue;
        const float* own = sm + csm_slot(z) * CSM_SLOT;
        const float dnr = own[SQ_DN * CSM_HN + hc];
        float d79;
        csm_collide(own, sm + csm_slot(z - 1) * CSM_SLOT, sm + csm_slot(z + 1) * CSM_SLOT, hc,
                    (1.f - om) / store_scale<T>(), dnr, bb, v, d79);
        float ux, uy, uz;
        const float dn = pull_finish<T>([&](int i) { return pop_at(pout, P, i, idx); }, v, d79, dnr, ux, uy, uz);
        put_fields(P, io, x, y, z, dn, ux, uy, uz, status);
    }
}

// Narrow grids (below one 32 x 4 tile): the same pass with one thread per
// node and no staging; every source's quantities are formed where they are
// used, by the same code as the staged ones, so both kernels give identical
// results.
template <typename T, bool IP>
__global__ void __launch_bounds__(128) k_pull_node(Params P, const T* pin, T* pout, CsmIO io,
                                                   const float4* __restrict__ F, int* status)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P.g.N) return;
    const Geom& g = P.g;
    int x, y, z;
    decompose(g, idx, x, y, z);
    const int s = slit_of(P, z);
    if (s < 0 || frozen(P, s)) return;
    const int zlo = P.sl[s].zlo, zhi = P.sl[s].zhi;
    const float om = P.sl[s].inv_tau, om1s = (1.f - om) / store_scale<T>();
    const bool shifted = P.shifted != 0;
    float v[Q];
    unsigned bb = 0;
    IpSlots q;
    if constexpr (IP) q = ip_slots(P, P.sl[s], s, x, y, z);
    csm_pull<0, Q, IP>(P, pin, idx, x, y, z, zlo, zhi, v, bb, q);
    const int p = pidx(g, x, y, z);
    float own[CSM_NF];
    src_terms(__ldg(io.dn + p), __ldg(io.ux + p), __ldg(io.uy + p), __ldg(io.uz + p), __ldg(F + idx), om, shifted,
              [&](int j, float val) { own[j] = val; });
    const float dnr = own[SQ_DN];
    // the source quantities of direction i, formed where they are used
    // (padded fields through their periodic images, the force at its
    // wrapped node); walls never ask (they use own)
    auto terms = [&](auto ic, float* out) {
        constexpr int i = decltype(ic)::value;
        int sx = x - kCx(i), sy = y - kCy(i), sz = z - kCz(i);
        sx = sx < 0 ? sx + g.nx : (sx >= g.nx ? sx - g.nx : sx);
        sy = sy < 0 ? sy + g.ny : (sy >= g.ny ? sy - g.ny : sy);
        if (g.zper) sz = sz < 0 ? sz + g.nz : (sz >= g.nz ? sz - g.nz : sz);
        const int ps = p - P.nbr[i];
        src_terms(__ldg(io.dn + ps), __ldg(io.ux + ps), __ldg(io.uy + ps), __ldg(io.uz + ps),
                  __ldg(F + (((long long)sz * g.ny + sy) * g.nx + sx)), om, shifted,
                  [&](int j, float val) { out[j] = val; });
    };
    auto wall = [&](int i) { return ((bb >> i) & 1u) != 0u; };
    auto diff = [&](auto ic, auto ipc) {
        constexpr int i = decltype(ic)::value, ip = decltype(ipc)::value;
        if (wall(i)) return mirror_diff<i, ip, 1>(own, own, v[i], v[ip], om1s, true);
        float a[CSM_NF], b[CSM_NF];
        terms(ic, a);
        terms(ipc, b);
        return mirror_diff<i, ip, 1>(a, b, v[i], v[ip], om1s, false);
    };
    using std::integral_constant;
    const float d7_10 = diff(integral_constant<int, 7>{}, integral_constant<int, 10>{});
    const float d9_8 = diff(integral_constant<int, 9>{}, integral_constant<int, 8>{});
    const float d10_8 = diff(integral_constant<int, 10>{}, integral_constant<int, 8>{});
    const float d79 = diff(integral_constant<int, 7>{}, integral_constant<int, 9>{});
    v[7] = d7_10;
    v[9] = d9_8;
    v[10] = d10_8;
    v[1] = diff(integral_constant<int, 1>{}, integral_constant<int, 2>{});
    v[3] = diff(integral_constant<int, 3>{}, integral_constant<int, 4>{});
    v[11] = diff(integral_constant<int, 11>{}, integral_constant<int, 14>{});
    v[13] = diff(integral_constant<int, 13>{}, integral_constant<int, 12>{});
    v[15] = diff(integral_constant<int, 15>{}, integral_constant<int, 18>{});
    v[17] = diff(integral_constant<int, 17>{}, integral_constant<int, 16>{});
    auto one = [&](auto ic) {
        constexpr int i = decltype(ic)::value;
        if constexpr (i == 0 || i == 2 || i == 4 || i == 5 || i == 6 || i == 8 || i == 12 || i == 14 || i == 16 ||
                      i == 18) {
            const bool w = i != 0 && wall(i);
            if (i == 0 || w) {
                v[i] = arrive<i, 1>(own, v[i], om1s, dnr, w);
            } else {
                float sv[CSM_NF];
                terms(ic, sv);
                v[i] = arrive<i, 1>(sv, v[i], om1s, dnr, false);
            }
        }
    };
    for_dirs(one);
    float ux, uy, uz;
    const float dn = IP ? pull_finish<T>([&](int i) { return pop_at_ip(pout, P, i, q.slot(i)); }, v, d79, dnr, ux,
                                         uy, uz)
                        : pull_finish<T>([&](int i) { return pop_at(pout, P, i, idx); }, v, d79, dnr, ux, uy, uz);
    put_fields(P, io, x, y, z, dn, ux, uy, uz, status);
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

cudaError_t launch_init_noise(const Params& P, float* dn, uint64_t seed, double amp, long long offset,
                              cudaStream_t s)
{
    k_init_noise<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, dn, seed, amp, offset);
    return cudaGetLastError();
}

cudaError_t launch_init_profiles(const Params& P, float* const f[4], const float* n_z, const float* ux_z,
                                 int hmax, cudaStream_t s)
{
    k_init_profiles<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, f[0], f[1], f[2], f[3], n_z, ux_z, hmax);
    return cudaGetLastError();
}

cudaError_t launch_init_fields(const Params& P, float* const f[4], const float* rho, const float* u,
                               cudaStream_t s)
{
    k_init_fields<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, f[0], f[1], f[2], f[3], rho, u);
    return cudaGetLastError();
}

cudaError_t launch_tick(const Params& P, int4* clk, cudaStream_t s)
{
    k_tick<<<nblocks(P.nslits, 128), 128, 0, s>>>(P, clk);
    return cudaGetLastError();
}

cudaError_t launch_pop_canon(const Params& P, void* pop, int i, void* canon, int to_pop, cudaStream_t s)
{
    if (P.storage == LBIF_STORE_F16)
        k_pop_canon<__half><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (__half*)pop, i, (__half*)canon, to_pop);
    else
        k_pop_canon<float><<<nblocks(P.g.N, 256), 256, 0, s>>>(P, (float*)pop, i, (float*)canon, to_pop);
    return cudaGetLastError();
}

cudaError_t launch_write_fields(const Params& P, const float* src, float* const f[4], cudaStream_t s)
{
    k_write_fields<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, src, f[0], f[1], f[2], f[3]);
    return cudaGetLastError();
}

cudaError_t launch_read_fields(const Params& P, const float* const f[4], float* out, cudaStream_t s)
{
    k_read_fields<<<nblocks(P.g.N, 256), 256, 0, s>>>(P, f[0], f[1], f[2], f[3], out);
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

bool csm_ok(const Geom& g) { return g.nx >= CSM_TX && g.ny >= CSM_TY; }

template <typename T, bool PF, bool IP>
static cudaError_t csm_tiled(const Params& P, const void* pin, void* pout, const CsmIO& io, const float4* F,
                             int* status, int lz, cudaStream_t s)
{
    const Geom& g = P.g;
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
        e = cudaFuncSetAttribute(k_csm<T, PF, IP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    k_csm<T, PF, IP><<<(unsigned)blocks, CSM_THREADS, smem, s>>>(P, (const T*)pin, (T*)pout, io, F, lz, tx, ty, status);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t csm_tma(const Params& P, const CUtensorMap* pmap, const void* pin, void* pout, const CsmIO& io,
                           const float4* F, int* status, int lz, cudaStream_t s)
{
    const Geom& g = P.g;
    const int tx = (g.nx + CSM_TX - 1) / CSM_TX, ty = (g.ny + CSM_TY - 1) / CSM_TY;
    const int segs = (g.nz + lz - 1) / lz;
    const long long blocks = (long long)tx * ty * segs;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    const size_t smem = csm_tma_smem_bytes<T>();
    static std::atomic<uint64_t> configured{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(k_csm_tma<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    k_csm_tma<T><<<(unsigned)blocks, CSM_THREADS, smem, s>>>(P, *pmap, (const T*)pin, (T*)pout, io, F, lz, tx, ty,
                                                            status);
    return cudaGetLastError();
}

cudaError_t launch_csm(const Params& P, const void* pin, void* pout, const CsmIO& io, const float4* F,
                       int* status, int lz, int prefetch, cudaStream_t s, const CUtensorMap* pmap)
{
    const Geom& g = P.g;
    const bool ip = P.inplace != 0, h16 = P.storage == LBIF_STORE_F16;
    if (prefetch == 2 && pmap && !ip && csm_ok(g)) {
        if (lz <= 0) lz = CSM_LZ;
        return h16 ? csm_tma<__half>(P, pmap, pin, pout, io, F, status, lz, s)
                   : csm_tma<float>(P, pmap, pin, pout, io, F, status, lz, s);
    }
    if (!csm_ok(g)) {
        const unsigned nb = nblocks(g.N, 128);
        if (h16 && ip) k_pull_node<__half, true><<<nb, 128, 0, s>>>(P, (const __half*)pin, (__half*)pout, io, F, status);
        if (h16 && !ip) k_pull_node<__half, false><<<nb, 128, 0, s>>>(P, (const __half*)pin, (__half*)pout, io, F, status);
        if (!h16 && ip) k_pull_node<float, true><<<nb, 128, 0, s>>>(P, (const float*)pin, (float*)pout, io, F, status);
        if (!h16 && !ip) k_pull_node<float, false><<<nb, 128, 0, s>>>(P, (const float*)pin, (float*)pout, io, F, status);
        return cudaGetLastError();
    }
    if (lz <= 0) lz = CSM_LZ;
    if (h16) {
        if (ip)
            return prefetch ? csm_tiled<__half, true, true>(P, pin, pout, io, F, status, lz, s)
                            : csm_tiled<__half, false, true>(P, pin, pout, io, F, status, lz, s);
        return prefetch ? csm_tiled<__half, true, false>(P, pin, pout, io, F, status, lz, s)
                        : csm_tiled<__half, false, false>(P, pin, pout, io, F, status, lz, s);
    }
    if (ip)
        return prefetch ? csm_tiled<float, true, true>(P, pin, pout, io, F, status, lz, s)
                        : csm_tiled<float, false, true>(P, pin, pout, io, F, status, lz, s);
    return prefetch ? csm_tiled<float, true, false>(P, pin, pout, io, F, status, lz, s)
                    : csm_tiled<float, false, false>(P, pin, pout, io, F, status, lz, s);
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
