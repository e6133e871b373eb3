// Host side of the C ABI declared in include/lbif.h: argument checks, the
// quadrature / tail tables (built in FP64, rounded once to FP32), the slit
// tables, device allocation, the per-step launch sequence, the ensemble
// driver (CUDA graph of K steps, per-slit FP64 residual, freezing) and its
// launch-shape autotuner.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include <mutex>

#include "lbif_internal.h"

using namespace lbif;

struct SlitDesc {
    int zlo, zhi;
    double eta, tau, body[3];
};

struct lbif_ctx {
    Params P;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* pop[2] = {nullptr, nullptr};
    int cur = 0;                      // populations of the current step
    float* dn[2] = {nullptr, nullptr};
    float* u[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    int fcur = 0;                     // dn[fcur], u[fcur]: the moments of step t (pop[cur] refers to them)
    int csm_lz = 0;                   // z planes per CTA of the pull pass (0 = default)
    int csm_pf = 0;                   // pull-pass gathers: 0 plain, 1 prefetched, 2 TMA boxes (autotuner)
    float* dG = nullptr;
    float4* Ft = nullptr;
    float4* F = nullptr;              // F / n0 per node (force kernel -> collision kernel)
    int* tail_off = nullptr;
    float4* tail_K = nullptr;
    int tail_pairs = 0;
    float2* tail_work = nullptr;      // spectral tail: fields, kernel transform, twiddles
    int tail_D = 0;                   // z reach of the tail kernel (planes)
    bool tail_fft = false;
    int* status_d = nullptr;
    int4* clk_d = nullptr;            // in place: per slit clock (t mod nx, ny, R)
    double* prof_d = nullptr;
    float* scratch = nullptr;         // 3 N floats, for host-side outputs
    SlitParam* d_sl = nullptr;
    int* d_zslit = nullptr;
    int* d_done = nullptr;
    std::vector<SlitParam> sl;
    std::vector<int> zslit;
    std::vector<int> done;
    bool batch = false;
    int ball_want = 0, force_group = 0;  // launch shapes (0 = defaults; set by the autotuner)
    CUtensorMap ball_map[2];             // tensor maps of dn[0..1] for the ball kernel's tiles
    bool ball_map_ok = false;
    CUtensorMap pop_map[2];              // tensor maps of pop[0..1] for the pull pass's source boxes
    bool pop_map_ok = false;
    bool ball_tma = true;                // stage the ball tiles with the maps (autotuner's choice)
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    int graph_state = -1;             // buffer indices the graph was captured from
    int64_t t = 0;
    int64_t G_t = -1, tail_t = -1;    // step the cached g2 field / tail force belong to
    std::vector<double> last_n, last_ux;
    int64_t last_t = -1;
    int sticky = 0;
    std::string err;
};

static thread_local std::string g_err = "no error";

static int fail(lbif_ctx* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    g_err = msg;
    return code;
}

#define CK(h, call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((h), LBIF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static size_t pop_bytes(const Params& P) { return (P.storage == LBIF_STORE_F16 ? 2 : 4); }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); NULL if the driver does not provide it.
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// 3-D map (x, y, z of the padded grid, FP32) of a padded field, with the
// ball kernel's plane tile as its box; out-of-range elements read as zero.
static bool make_ball_map(const Geom& g, int sigma, float* base, CUtensorMap* out)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    int W, H;
    ball_box(sigma, &W, &H);
    if (W > 256 || H > 256 || (W * 4) % 16) return false;
    cuuint64_t dims[3] = {(cuuint64_t)g.px, (cuuint64_t)g.py, (cuuint64_t)g.pz};
    cuuint64_t strides[2] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.px * g.py * 4};
    cuuint32_t box[3] = {(cuuint32_t)W, (cuuint32_t)H, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 4-D map (x, y, z, direction) of a two-buffer population array, with the
// pull pass's per-direction source box; false where the layout does not
// allow one (rows not a multiple of 16 bytes, grids narrower than a box).
static bool make_pop_map(const Params& P, void* base, CUtensorMap* out)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    const Geom& g = P.g;
    if (!enc || P.inplace || !csm_ok(g)) return false;
    const int es = P.storage == LBIF_STORE_F16 ? 2 : 4;
    int W, H;
    pop_box(P.storage, &W, &H);
    if (((long long)g.nx * es) % 16 || ((long long)g.Npad * es) % 16 || g.nx < W || g.ny < H + 2) return false;
    cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)Q};
    cuuint64_t strides[3] = {(cuuint64_t)g.nx * es, (cuuint64_t)g.nx * g.ny * es, (cuuint64_t)g.Npad * es};
    cuuint32_t box[4] = {(cuuint32_t)W, (cuuint32_t)H, 1, 1};
    cuuint32_t ests[4] = {1, 1, 1, 1};
    return enc(out, es == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims,
               strides, box, ests, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the map of the population buffer the pull pass reads (pop[i]), or NULL
static const CUtensorMap* pop_map(const lbif_ctx* h, int i)
{
    return h->pop_map_ok ? &h->pop_map[i] : nullptr;
}

// the map of the buffer the ball kernel reads (dn[i]), or NULL
static const CUtensorMap* ball_map(const lbif_ctx* h, int i)
{
    return h->ball_map_ok && h->ball_tma ? &h->ball_map[i] : nullptr;
}

// tail force of the density field dn: spectral in x, y when available
static cudaError_t run_tail(lbif_ctx* h, const float* dn)
{
    if (h->tail_fft) return launch_tail_spectral(h->P, dn, h->tail_D, h->tail_work, h->Ft, h->stream);
    return launch_tail(h->P, dn, h->tail_off, h->tail_K, h->tail_pairs, h->Ft, h->stream);
}

// padded fields carry PAD_SLACK floats before their first element
static cudaError_t padded_alloc(size_t P, float** out)
{
    float* raw = nullptr;
    *out = nullptr;
    const cudaError_t e = cudaMalloc((void**)&raw, sizeof(float) * (P + 2 * PAD_SLACK));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    *out = raw + PAD_SLACK;
    return cudaSuccess;
}

// a failed device allocation during creation: LBIF_ERR_NOMEM when the device
// is out of memory, LBIF_ERR_CUDA with the runtime's message otherwise (no
// device, a broken context)
static int alloc_failed(cudaError_t e)
{
    if (e == cudaErrorMemoryAllocation) return fail(nullptr, LBIF_ERR_NOMEM, "create: device allocation failed");
    return fail(nullptr, LBIF_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e));
}

static void padded_free(float* p)
{
    if (p) cudaFree(p - PAD_SLACK);
}

static void free_ctx(lbif_ctx* h)
{
    if (!h) return;
    if (h->graph) cudaGraphExecDestroy(h->graph);
    void* bufs[] = {h->pop[0], h->pop[1], h->Ft, h->F, h->tail_off, h->tail_K, h->tail_work, h->status_d,
                    h->prof_d, h->scratch, h->d_sl, h->d_zslit, h->d_done, h->clk_d};
    for (void* b : bufs)
        if (b) cudaFree(b);
    float* pads[] = {h->dn[0], h->dn[1], h->u[0][0], h->u[0][1], h->u[0][2],
                     h->u[1][0], h->u[1][1], h->u[1][2], h->dG};
    for (float* q : pads) padded_free(q);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

static Fields fields_of(const lbif_ctx* h)
{
    Fields f;
    f.dn = h->dn[h->fcur];
    f.ux = h->u[h->fcur][0];
    f.uy = h->u[h->fcur][1];
    f.uz = h->u[h->fcur][2];
    f.dG = h->dG;
    return f;
}

// the padded fields dn, ux, uy, uz of buffer set k
static void field_set(lbif_ctx* h, int k, float* out[4])
{
    out[0] = h->dn[k];
    out[1] = h->u[k][0];
    out[2] = h->u[k][1];
    out[3] = h->u[k][2];
}

static void invalidate(lbif_ctx* h) { h->G_t = h->tail_t = -1; }

// --------------------------------------------------------------------------
// tables
// --------------------------------------------------------------------------
static int padded_offset(const Geom& g, int dx, int dy, int dz)
{
    return (dz * g.py + dy) * g.px + dx;
}

// 18-point sphere rule: 6 axis points (weight 1/30) and the 12 face
// diagonals (weight 1/15), layout in lbif_internal.h. The off-lattice
// points sit at sigma/sqrt2 (neighbour) and sigma/(2 sqrt2) (midpoint) along
// two axes; linear interpolation between floor and floor + 1 on each.
static int build_shell(Params& P)
{
    const Geom& g = P.g;
    for (int a = 0; a < 3; ++a) {
        int e[3] = {0, 0, 0};
        e[a] = 1;
        P.sh.ax_nb[a] = padded_offset(g, P.sigma * e[0], P.sigma * e[1], P.sigma * e[2]);
        int hh = P.sigma / 2;
        P.sh.ax_md[a] = padded_offset(g, hh * e[0], hh * e[1], hh * e[2]);
    }
    const int stride[3] = {1, g.px, g.px * g.py};
    const int planes[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    const double A = P.sigma / sqrt(2.0);
    for (int pl = 0; pl < 3; ++pl) {
        int sa = stride[planes[pl][0]], sb = stride[planes[pl][1]];
        for (int which = 0; which < 2; ++which) {
            double s = which ? 0.5 * A : A;
            int lo = (int)floor(s);
            double t = s - lo;
            if (t <= 1e-12 || t >= 1.0 - 1e-12) return -1;  // irrational for every even sigma
            for (int k = 0; k < 4; ++k) {
                int ka = k & 1, kb = k >> 1;
                float w = (float)((ka ? t : 1.0 - t) * (kb ? t : 1.0 - t));
                if (which) {
                    P.sh.md_a[pl][k] = (lo + ka) * sa;
                    P.sh.md_b[pl][k] = (lo + kb) * sb;
                    P.sh.md_w[pl][k] = w;
                } else {
                    P.sh.nb_a[pl][k] = (lo + ka) * sa;
                    P.sh.nb_b[pl][k] = (lo + kb) * sb;
                    P.sh.nb_w[pl][k] = w;
                }
            }
        }
    }
    return 0;
}

static int ball_count(int sigma)
{
    int r = sigma / 2, c = 0;
    for (int dz = -r; dz <= r; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx)
                if (dx * dx + dy * dy + dz * dz <= r * r) ++c;
    return c;
}

static double g2_host(double e, int form)
{
    double d = (1 - e) * (1 - e) * (1 - e);
    return form == 1 ? (1 - 0.5 * e) / d : (1 - 0.5 * e + 0.25 * e * e) / d;
}

static SlitParam slit_param(const SlitDesc& d, double sigma, int g2form)
{
    const double kT = 1.0 / 3.0;
    double n0 = 6.0 * d.eta / (M_PI * sigma * sigma * sigma);
    SlitParam s;
    memset(&s, 0, sizeof(s));
    s.rho0 = (float)n0;
    s.eta0 = (float)d.eta;
    s.G0 = (float)g2_host(d.eta, g2form);
    s.inv_tau = (float)(1.0 / d.tau);
    s.hs_pref = (float)(-kT * sigma * sigma * 4.0 * M_PI * n0);
    s.p_pref = (float)(kT * sigma * sigma * sigma / 6.0 * 4.0 * M_PI * n0 * n0);
    for (int a = 0; a < 3; ++a) s.body[a] = (float)d.body[a];
    s.zlo = d.zlo;
    s.zhi = d.zhi;
    return s;
}

// --------------------------------------------------------------------------
// create / destroy
// --------------------------------------------------------------------------
static int check_common(double sigma, const lbif_force& F, const lbif_opts& O, const char* who)
{
    std::string w(who);
    if (!(sigma >= 2.0) || sigma != floor(sigma) || ((int)sigma) % 2 != 0 || sigma > MAX_SIGMA)
        return fail(nullptr, LBIF_ERR_UNSUPPORTED,
                    w + ": sigma must be an even integer in [2, 24] lattice spacings");
    if (O.storage != LBIF_STORE_F32 && O.storage != LBIF_STORE_F16)
        return fail(nullptr, LBIF_ERR_ARG, w + ": storage must be 0 (FP32) or 1 (FP16)");
    if (!(O.noise >= 0.0 && O.noise < 1.0)) return fail(nullptr, LBIF_ERR_ARG, w + ": noise must be in [0,1)");
    if (F.tail && !(F.rcut >= 1.0 && F.rcut <= 4.0 && F.eps >= 0.0))
        return fail(nullptr, LBIF_ERR_ARG, w + ": tail needs rcut in [1,4] and eps >= 0");
    if ((F.g2_form != 0 && F.g2_form != 1)) return fail(nullptr, LBIF_ERR_ARG, w + ": g2_form must be 0 or 1");
    if (F.c2 != 0 && F.c2 != 1) return fail(nullptr, LBIF_ERR_ARG, w + ": c2 must be 0 or 1");
    if (F.shifted != 0 && F.shifted != 1) return fail(nullptr, LBIF_ERR_ARG, w + ": shifted must be 0 or 1");
    if (F.shifted && F.c2)
        return fail(nullptr, LBIF_ERR_UNSUPPORTED, w + ": the shifted forcing does not add the energy source");
    for (int a = 0; a < 3; ++a)
        if (!isfinite(F.body[a])) return fail(nullptr, LBIF_ERR_ARG, w + ": body force not finite");
    return LBIF_OK;
}

static int create_impl(lbif_handle* out, int nx, int ny, int nz, int sigma, int zper,
                       const lbif_force& F, const lbif_opts& O, const std::vector<SlitDesc>& slits,
                       const std::vector<int>& zslit, bool batch)
{
    lbif_ctx* h = new lbif_ctx();
    memset(&h->P, 0, sizeof(Params));
    Params& P = h->P;
    Geom& g = P.g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.zper = zper;
    g.hw = sigma;
    if (F.tail) g.hw = std::max(g.hw, (int)ceil(F.rcut * sigma));
    g.hw = (g.hw + 3) / 4 * 4;                   // rows 16-byte aligned
    g.px = (g.nx + 2 * g.hw + 8 + 3) / 4 * 4;    // + slack columns for float4 windows
    g.py = g.ny + 2 * g.hw;
    g.pz = g.nz + 2 * g.hw;
    g.N = (long long)g.nx * g.ny * g.nz;
    g.Npad = (g.N + 63) / 64 * 64;
    long long ring_planes = 0;  // in place: every slit's ring of storage planes
    std::vector<int> ring_base;
    for (const SlitDesc& d : slits) {
        ring_base.push_back((int)ring_planes);
        ring_planes += (d.zhi - d.zlo + 1) + (zper ? 0 : 1);
    }
    if (O.inplace) g.Npad = ((long long)g.nx * g.ny * ring_planes + 63) / 64 * 64;
    g.P = (long long)g.px * g.py * g.pz;
    if (g.P >= (1LL << 31) || g.Npad >= (1LL << 31)) {
        delete h;
        return fail(nullptr, LBIF_ERR_UNSUPPORTED, "create: padded grid exceeds 2^31 nodes");
    }
    if (O.inplace && (long long)Q * g.Npad >= (1LL << 32)) {
        delete h;
        return fail(nullptr, LBIF_ERR_UNSUPPORTED,
                    "create: the in-place layout holds at most 2^32 population elements (use two buffers)");
    }
    const double kT = 1.0 / 3.0;
    P.sigma = sigma;
    P.kappa = (float)(2.0 / (sqrt(kT) * sqrt(M_PI)));
    P.inv_sigma = (float)(1.0 / sigma);
    P.ball_inv = (float)(1.0 / ball_count(sigma));
    P.hs = F.hs ? 1 : 0;
    P.coupling = F.coupling ? 1 : 0;
    P.regularize = F.regularize ? 1 : 0;
    P.g2form = F.g2_form;
    P.tail = F.tail ? 1 : 0;
    P.c2 = F.c2 ? 1 : 0;
    P.shifted = F.shifted ? 1 : 0;
    P.storage = O.storage;
    P.inplace = O.inplace ? 1 : 0;
    P.nslits = (int)slits.size();
    {
        const int cx[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        const int cy[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        const int cz[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        for (int i = 0; i < Q; ++i) {
            P.nbr[i] = padded_offset(g, cx[i], cy[i], cz[i]);
            P.soff[i] = cx[i] + (long long)cy[i] * g.nx + (long long)cz[i] * g.nx * g.ny;
            P.dbase[i] = (long long)i * g.Npad;
            P.doff[i] = P.dbase[i] - P.soff[i];
            P.dbase32[i] = O.inplace ? (unsigned)P.dbase[i] : 0u;
        }
    }
    if (build_shell(P)) {
        delete h;
        return fail(nullptr, LBIF_ERR_UNSUPPORTED, "create: quadrature tables do not fit");
    }
    h->batch = batch;
    for (size_t k = 0; k < slits.size(); ++k) {
        SlitParam sp = slit_param(slits[k], sigma, F.g2_form);
        sp.zb = ring_base[k];
        sp.R = (slits[k].zhi - slits[k].zlo + 1) + (zper ? 0 : 1);
        h->sl.push_back(sp);
    }
    h->zslit = zslit;
    h->done.assign(slits.size(), 0);
    if (O.stream) {
        h->stream = (cudaStream_t)O.stream;
    } else if (batch) {
        // graph capture needs a stream other than the legacy default one
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return fail(nullptr, LBIF_ERR_CUDA, "create: stream creation failed");
        }
        h->own_stream = true;
    }

    // tail taps: one representative of each +-d pair with sigma <= |d| <= rcut sigma
    std::vector<int> toff, tdx, tdy, tdz;
    std::vector<float4> tK;
    if (P.tail) {
        double rmax = F.rcut * sigma;
        int R = (int)ceil(rmax);
        h->tail_D = R;
        double s6 = pow((double)sigma, 6.0), s12 = s6 * s6;
        for (int dz = 0; dz <= R; ++dz)
            for (int dy = (dz == 0 ? 0 : -R); dy <= R; ++dy)
                for (int dx = ((dz == 0 && dy == 0) ? 1 : -R); dx <= R; ++dx) {
                    double r2 = (double)dx * dx + (double)dy * dy + (double)dz * dz;
                    if (r2 < (double)sigma * sigma || r2 > rmax * rmax) continue;
                    double r = sqrt(r2);
                    double dphi = 4.0 * F.eps * (-12.0 * s12 / pow(r, 13.0) + 6.0 * s6 / pow(r, 7.0));
                    toff.push_back(padded_offset(g, dx, dy, dz));
                    tdx.push_back(dx);
                    tdy.push_back(dy);
                    tdz.push_back(dz);
                    tK.push_back(make_float4((float)(dphi * dx / r), (float)(dphi * dy / r),
                                             (float)(dphi * dz / r), 0.f));
                }
        h->tail_pairs = (int)toff.size();
    }

    size_t pb = pop_bytes(P) * (size_t)Q * (size_t)g.Npad;
#define ALLOC(ptr, bytes)                                                                   \
    do {                                                                                    \
        const cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));                         \
        if (e_ != cudaSuccess) {                                                            \
            cudaGetLastError();                                                             \
            free_ctx(h);                                                                    \
            return alloc_failed(e_);                                                        \
        }                                                                                   \
    } while (0)
    ALLOC(h->pop[0], pb);
    if (!P.inplace) ALLOC(h->pop[1], pb);
    h->pop_map_ok = !P.inplace && make_pop_map(P, h->pop[0], &h->pop_map[0]) &&
                    make_pop_map(P, h->pop[1], &h->pop_map[1]);
    ALLOC(h->clk_d, sizeof(int4) * h->sl.size());
    ALLOC(h->F, sizeof(float4) * (size_t)g.N);
    ALLOC(h->status_d, sizeof(int));
    ALLOC(h->prof_d, sizeof(double) * profile_doubles(g));
    ALLOC(h->d_sl, sizeof(SlitParam) * h->sl.size());
    ALLOC(h->d_zslit, sizeof(int) * (size_t)g.nz);
    ALLOC(h->d_done, sizeof(int) * h->sl.size());
    if (P.tail) {
        ALLOC(h->Ft, sizeof(float4) * (size_t)g.N);
        ALLOC(h->tail_off, sizeof(int) * toff.size());
        ALLOC(h->tail_K, sizeof(float4) * tK.size());
    }
#undef ALLOC
    {
        float** pads[] = {&h->dn[0], &h->dn[1], &h->u[0][0], &h->u[0][1], &h->u[0][2],
                          &h->u[1][0], &h->u[1][1], &h->u[1][2], &h->dG};
        for (float** q : pads) {
            const cudaError_t e = padded_alloc((size_t)g.P, q);
            if (e != cudaSuccess) {
                free_ctx(h);
                return alloc_failed(e);
            }
        }
        h->ball_map_ok = make_ball_map(g, P.sigma, h->dn[0], &h->ball_map[0]) &&
                         make_ball_map(g, P.sigma, h->dn[1], &h->ball_map[1]);
    }
    P.sl = h->d_sl;
    P.zslit = h->d_zslit;
    P.done = h->d_done;
    P.clk = h->clk_d;
    lbif_ctx* hc = h;
#define CKC(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            std::string m_ = std::string(#call) + ": " + cudaGetErrorString(e_);            \
            free_ctx(hc);                                                                   \
            return fail(nullptr, LBIF_ERR_CUDA, m_);                                        \
        }                                                                                   \
    } while (0)
    CKC(cudaMemcpyAsync(h->d_sl, h->sl.data(), sizeof(SlitParam) * h->sl.size(), cudaMemcpyHostToDevice,
                        h->stream));
    CKC(cudaMemcpyAsync(h->d_zslit, h->zslit.data(), sizeof(int) * h->zslit.size(),
                        cudaMemcpyHostToDevice, h->stream));
    CKC(cudaMemsetAsync(h->d_done, 0, sizeof(int) * h->sl.size(), h->stream));
    CKC(cudaMemsetAsync(h->pop[0], 0, pb, h->stream));
    if (h->pop[1]) CKC(cudaMemsetAsync(h->pop[1], 0, pb, h->stream));
    CKC(cudaMemsetAsync(h->clk_d, 0, sizeof(int4) * h->sl.size(), h->stream));
    {
        float* pads[] = {h->dn[0], h->dn[1], h->u[0][0], h->u[0][1], h->u[0][2],
                         h->u[1][0], h->u[1][1], h->u[1][2], h->dG};
        const float outside[] = {-1.f, -1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (float* q : pads)
            CKC(cudaMemsetAsync(q - PAD_SLACK, 0, sizeof(float) * ((size_t)g.P + 2 * PAD_SLACK), h->stream));
        CKC(launch_fill_outside(P, pads, outside, 9, h->stream));
        if (batch) {
            // gap planes between stacked slits hold the outside values too
            for (int z = 0; z < g.nz; ++z) {
                if (zslit[z] >= 0) continue;
                size_t plane = (size_t)g.px * g.py, off = (size_t)(z + g.hw) * plane;
                std::vector<float> minus1(plane, -1.f);
                for (float* d : h->dn)
                    CKC(cudaMemcpyAsync(d + off, minus1.data(), sizeof(float) * plane,
                                        cudaMemcpyHostToDevice, h->stream));
                CKC(cudaStreamSynchronize(h->stream));
            }
        }
    }
    CKC(cudaMemsetAsync(h->status_d, 0, sizeof(int), h->stream));
    if (P.tail) {
        CKC(cudaMemcpyAsync(h->tail_off, toff.data(), sizeof(int) * toff.size(),
                            cudaMemcpyHostToDevice, h->stream));
        // spectral path when the lateral extents allow it; else the direct sum
        if (tail_spectral_ok(g)) {
            if (cudaMalloc((void**)&h->tail_work, tail_spectral_bytes(g, h->tail_D)) == cudaSuccess &&
                tail_spectral_init(g, h->tail_D, tdx.data(), tdy.data(), tdz.data(), tK.data(), (int)tK.size(),
                                   h->zslit.data(), h->tail_work, h->stream) == cudaSuccess) {
                h->tail_fft = true;
            } else {
                cudaGetLastError();
                if (h->tail_work) cudaFree(h->tail_work);
                h->tail_work = nullptr;
            }
        }
        CKC(cudaMemcpyAsync(h->tail_K, tK.data(), sizeof(float4) * tK.size(),
                            cudaMemcpyHostToDevice, h->stream));
    }
    CKC(launch_init_noise(P, h->dn[0], O.seed, O.noise, 0, h->stream));
    CKC(cudaStreamSynchronize(h->stream));
#undef CKC
    *out = h;
    return LBIF_OK;
}

extern "C" int lbif_create(lbif_handle* out, lbif_grid gr, double sigma, double eta, double tau,
                           lbif_walls w, const lbif_force* f, const lbif_opts* o)
{
    if (!out) return fail(nullptr, LBIF_ERR_ARG, "lbif_create: out is NULL");
    *out = nullptr;
    if (gr.nx < 1 || gr.ny < 1 || gr.nz < 1)
        return fail(nullptr, LBIF_ERR_ARG, "lbif_create: grid extents must be >= 1");
    if (!(eta > 0.0 && eta < 1.0)) return fail(nullptr, LBIF_ERR_ARG, "lbif_create: eta must be in (0,1)");
    if (!(tau > 0.5)) return fail(nullptr, LBIF_ERR_ARG, "lbif_create: tau must be > 1/2");
    if (w.z != LBIF_WALL_BOUNCEBACK && w.z != LBIF_PERIODIC)
        return fail(nullptr, LBIF_ERR_ARG, "lbif_create: walls.z must be BOUNCEBACK or PERIODIC");
    lbif_force fz;
    memset(&fz, 0, sizeof(fz));
    const lbif_force& F = f ? *f : fz;
    lbif_opts oz;
    memset(&oz, 0, sizeof(oz));
    oz.noise = 1e-3;
    const lbif_opts& O = o ? *o : oz;
    int rc = check_common(sigma, F, O, "lbif_create");
    if (rc) return rc;
    SlitDesc d;
    d.zlo = 0;
    d.zhi = gr.nz - 1;
    d.eta = eta;
    d.tau = tau;
    for (int a = 0; a < 3; ++a) d.body[a] = F.body[a];
    std::vector<int> zs(gr.nz, 0);
    return create_impl(out, gr.nx, gr.ny, gr.nz, (int)sigma, w.z == LBIF_PERIODIC, F, O, {d}, zs, false);
}

extern "C" int lbif_batch_create(lbif_handle* out, int32_t nslits, const int32_t* H, const double* eta,
                                 const double* Fx, const double* tau, double sigma, int32_t nx,
                                 int32_t ny, const lbif_force* f, const lbif_opts* o)
{
    if (!out) return fail(nullptr, LBIF_ERR_ARG, "lbif_batch_create: out is NULL");
    *out = nullptr;
    if (nslits < 1 || !H || !eta || !Fx || !tau || nx < 1 || ny < 1)
        return fail(nullptr, LBIF_ERR_ARG, "lbif_batch_create: bad arguments");
    lbif_force fz;
    memset(&fz, 0, sizeof(fz));
    const lbif_force& F = f ? *f : fz;
    lbif_opts oz;
    memset(&oz, 0, sizeof(oz));
    oz.noise = 1e-3;
    const lbif_opts& O = o ? *o : oz;
    int rc = check_common(sigma, F, O, "lbif_batch_create");
    if (rc) return rc;
    int hw = (int)sigma;
    if (F.tail) hw = std::max(hw, (int)ceil(F.rcut * sigma));
    hw = (hw + 3) / 4 * 4;
    std::vector<SlitDesc> slits;
    std::vector<int> zs;
    for (int s = 0; s < nslits; ++s) {
        if (H[s] < 1 || !(eta[s] > 0.0 && eta[s] < 1.0) || !(tau[s] > 0.5) || !isfinite(Fx[s]))
            return fail(nullptr, LBIF_ERR_ARG, "lbif_batch_create: bad slit parameters");
        if (s > 0) zs.insert(zs.end(), hw, -1);  // gap of outside planes
        SlitDesc d;
        d.zlo = (int)zs.size();
        d.zhi = d.zlo + H[s] - 1;
        d.eta = eta[s];
        d.tau = tau[s];
        d.body[0] = Fx[s];
        d.body[1] = d.body[2] = 0.0;
        slits.push_back(d);
        zs.insert(zs.end(), H[s], s);
    }
    return create_impl(out, nx, ny, (int)zs.size(), (int)sigma, 0, F, O, slits, zs, true);
}

extern "C" int lbif_destroy(lbif_handle h)
{
    if (!h) return fail(nullptr, LBIF_ERR_ARG, "lbif_destroy: NULL handle");
    cudaStreamSynchronize(h->stream);
    free_ctx(h);
    return LBIF_OK;
}

extern "C" const char* lbif_last_error(lbif_handle h)
{
    if (h) return h->err.empty() ? "no error" : h->err.c_str();
    return g_err.c_str();
}

// --------------------------------------------------------------------------
// stepping
// --------------------------------------------------------------------------
// The g2 field and the tail force of the current moments, cached per step so
// that output calls between steps do not redo them. The moments themselves
// are always current: the pull pass writes those of the step it produces,
// and every state set from outside is an equilibrium whose moments are the
// given fields.
static int refresh_fields(lbif_ctx* h, bool want_G, int skip_done)
{
    const Params& P = h->P;
    float* dnow = h->dn[h->fcur];
    if (want_G && h->G_t != h->t) {
        CK(h, launch_ball(P, dnow, h->dG, h->status_d, h->ball_want, skip_done, h->stream, ball_map(h, h->fcur)));
        h->G_t = skip_done ? -1 : h->t;
    }
    if (P.tail && h->tail_t != h->t) {
        CK(h, run_tail(h, dnow));
        h->tail_t = skip_done ? -1 : h->t;
    }
    return LBIF_OK;
}

// collision, streaming and the new moments of step t -> t + 1 (force F of
// step t computed)
static int collide_stream(lbif_ctx* h)
{
    const Params& P = h->P;
    float* const* u = h->u[h->fcur];
    float* const* w = h->u[h->fcur ^ 1];
    CsmIO io{h->dn[h->fcur], u[0], u[1], u[2], h->dn[h->fcur ^ 1], w[0], w[1], w[2]};
    if (P.inplace) {
        CK(h, launch_csm(P, h->pop[0], h->pop[0], io, h->F, h->status_d, h->csm_lz, h->csm_pf, h->stream));
        CK(h, launch_tick(P, h->clk_d, h->stream));
    } else {
        CK(h, launch_csm(P, h->pop[h->cur], h->pop[h->cur ^ 1], io, h->F, h->status_d, h->csm_lz, h->csm_pf,
                         h->stream, pop_map(h, h->cur)));
        h->cur ^= 1;
    }
    h->fcur ^= 1;
    h->t += 1;
    return LBIF_OK;
}

static int advance(lbif_ctx* h)
{
    const Params& P = h->P;
    const Fields f = fields_of(h);
    CK(h, launch_force(P, f, h->Ft, h->F, h->force_group, h->stream));
    return collide_stream(h);
}

// one full step of the active slits (frozen slits skipped)
static int one_step(lbif_ctx* h)
{
    int rc = refresh_fields(h, h->P.hs != 0, 1);
    if (rc) return rc;
    return advance(h);
}

extern "C" int lbif_step(lbif_handle h, int64_t nsteps)
{
    if (!h || nsteps < 0) return fail(h, LBIF_ERR_ARG, "lbif_step: bad arguments");
    for (int64_t k = 0; k < nsteps; ++k) {
        int rc = one_step(h);
        if (rc) return rc;
    }
    return LBIF_OK;
}

extern "C" int lbif_step_profiled(lbif_handle h, int64_t nsteps, double* kernel_ms,
                                  int64_t* launches, int32_t nk)
{
    if (!h || nsteps < 0 || !kernel_ms || !launches || nk < 5)
        return fail(h, LBIF_ERR_ARG, "lbif_step_profiled: bad arguments");
    const Params& P = h->P;
    for (int k = 0; k < nk; ++k) {
        kernel_ms[k] = 0.0;
        launches[k] = 0;
    }
    int per = 2 + (P.hs ? 1 : 0) + (P.tail ? 1 : 0);
    std::vector<cudaEvent_t> ev((size_t)nsteps * per + 1);
    std::vector<int> cls((size_t)nsteps * per);
    for (auto& e : ev) CK(h, cudaEventCreate(&e));
    size_t j = 0;
    CK(h, cudaEventRecord(ev[0], h->stream));
    for (int64_t s = 0; s < nsteps; ++s) {
        // the same launches as one_step, each timed
        float* dnew = h->dn[h->fcur];
        const Fields f = fields_of(h);
        if (P.hs) {
            CK(h, launch_ball(P, dnew, h->dG, h->status_d, h->ball_want, 1, h->stream, ball_map(h, h->fcur)));
            cls[j] = 1;
            CK(h, cudaEventRecord(ev[++j], h->stream));
        }
        if (P.tail) {
            CK(h, run_tail(h, dnew));
            cls[j] = 2;
            CK(h, cudaEventRecord(ev[++j], h->stream));
        }
        CK(h, launch_force(P, f, h->Ft, h->F, h->force_group, h->stream));
        cls[j] = 3;
        CK(h, cudaEventRecord(ev[++j], h->stream));
        int rc = collide_stream(h);
        if (rc) return rc;
        cls[j] = 4;
        CK(h, cudaEventRecord(ev[++j], h->stream));
    }
    h->G_t = h->tail_t = -1;
    CK(h, cudaEventSynchronize(ev[j]));
    for (size_t k = 0; k < j; ++k) {
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
        kernel_ms[cls[k]] += ms;
        launches[cls[k]] += 1;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return LBIF_OK;
}

static int check_status(lbif_ctx* h)
{
    int st = 0;
    CK(h, cudaMemcpyAsync(&st, h->status_d, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (st) h->sticky |= st;
    if (h->sticky & 4) return fail(h, LBIF_ERR_TIMEOUT, "a bounded device wait for a tile copy ran out");
    if (h->sticky)
        return fail(h, LBIF_ERR_DIVERGED,
                    (h->sticky & 2) ? "state diverged: coarse-grained packing fraction reached 1"
                                    : "state diverged: non-finite or non-positive density");
    return LBIF_OK;
}

// 4 N floats: host-side outputs and inputs (a density and a velocity field,
// the four moment fields of a checkpoint)
static int ensure_scratch(lbif_ctx* h)
{
    if (h->scratch) return LBIF_OK;
    if (cudaMalloc((void**)&h->scratch, sizeof(float) * 4 * (size_t)h->P.g.N) != cudaSuccess) {
        cudaGetLastError();
        h->scratch = nullptr;
        return fail(h, LBIF_ERR_NOMEM, "scratch allocation failed");
    }
    return LBIF_OK;
}

extern "C" int lbif_moments(lbif_handle h, float* rho, float* u, float* pressure, int32_t on_device)
{
    if (!h) return fail(nullptr, LBIF_ERR_ARG, "lbif_moments: NULL handle");
    const Params& P = h->P;
    int rc = refresh_fields(h, pressure && P.hs, 0);
    if (rc) return rc;
    size_t N = (size_t)P.g.N;
    if (on_device) {
        CK(h, launch_moments_out(P, fields_of(h), rho, u, pressure, h->stream));
    } else {
        if ((rc = ensure_scratch(h))) return rc;
        float* d = h->scratch;
        if (rho) {
            CK(h, launch_moments_out(P, fields_of(h), d, nullptr, nullptr, h->stream));
            CK(h, cudaMemcpyAsync(rho, d, sizeof(float) * N, cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
        }
        if (pressure) {
            CK(h, launch_moments_out(P, fields_of(h), nullptr, nullptr, d, h->stream));
            CK(h, cudaMemcpyAsync(pressure, d, sizeof(float) * N, cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
        }
        if (u) {
            CK(h, launch_moments_out(P, fields_of(h), nullptr, d, nullptr, h->stream));
            CK(h, cudaMemcpyAsync(u, d, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, h->stream));
        }
    }
    return check_status(h);
}

extern "C" int lbif_forces(lbif_handle h, float* F, int32_t on_device)
{
    if (!h || !F) return fail(h, LBIF_ERR_ARG, "lbif_forces: bad arguments");
    const Params& P = h->P;
    int rc = refresh_fields(h, P.hs != 0, 0);
    if (rc) return rc;
    // the same force kernel as the time step, then a layout change to SoA
    CK(h, launch_force(P, fields_of(h), h->Ft, h->F, h->force_group, h->stream));
    if (on_device) {
        CK(h, launch_force_soa(P, h->F, F, h->stream));
    } else {
        if ((rc = ensure_scratch(h))) return rc;
        CK(h, launch_force_soa(P, h->F, h->scratch, h->stream));
        CK(h, cudaMemcpyAsync(F, h->scratch, sizeof(float) * 3 * (size_t)P.g.N,
                              cudaMemcpyDeviceToHost, h->stream));
    }
    return check_status(h);
}

static void reset_time(lbif_ctx* h)
{
    h->t = 0;
    h->last_t = -1;
    invalidate(h);
}

// every stored population of the current state 0 (an equilibrium; in place,
// the slits' clocks restart)
static int zero_populations(lbif_ctx* h)
{
    const size_t pb = pop_bytes(h->P) * (size_t)Q * (size_t)h->P.g.Npad;
    CK(h, cudaMemsetAsync(h->pop[h->cur], 0, pb, h->stream));
    CK(h, cudaMemsetAsync(h->clk_d, 0, sizeof(int4) * h->sl.size(), h->stream));
    return LBIF_OK;
}

extern "C" int lbif_set_fields(lbif_handle h, const float* rho, const float* u, int32_t on_device)
{
    if (!h || !rho) return fail(h, LBIF_ERR_ARG, "lbif_set_fields: bad arguments");
    const Params& P = h->P;
    size_t N = (size_t)P.g.N;
    const float* drho = rho;
    const float* du = u;
    if (!on_device) {
        int rc = ensure_scratch(h);
        if (rc) return rc;
        float* d = h->scratch;
        CK(h, cudaMemcpyAsync(d, rho, sizeof(float) * N, cudaMemcpyHostToDevice, h->stream));
        drho = d;
        if (u) {
            CK(h, cudaMemcpyAsync(d + N, u, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, h->stream));
            du = d + N;
        }
    }
    // the equilibrium of the given fields: stored non-equilibrium parts 0,
    // the fields themselves are its moments (no moments pass)
    int rc = zero_populations(h);
    if (rc) return rc;
    float* f[4];
    field_set(h, h->fcur, f);
    CK(h, launch_init_fields(P, f, drho, du, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    reset_time(h);
    return LBIF_OK;
}

// FP64 per-plane sums of the current state (all slits, frozen ones included)
static int plane_sums(lbif_ctx* h, std::vector<double>& prof)
{
    const Params& P = h->P;
    int rc = refresh_fields(h, false, 0);
    if (rc) return rc;
    CK(h, launch_profiles(P, fields_of(h), h->prof_d, h->stream));
    prof.resize((size_t)P.g.nz * 5);
    CK(h, cudaMemcpyAsync(prof.data(), h->prof_d, sizeof(double) * prof.size(),
                          cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBIF_OK;
}

extern "C" int lbif_profiles(lbif_handle h, double* n_z, double* ux_z, double* out4)
{
    if (!h) return fail(nullptr, LBIF_ERR_ARG, "lbif_profiles: NULL handle");
    const Params& P = h->P;
    std::vector<double> prof;
    int rc = plane_sums(h, prof);
    if (rc) return rc;
    double A = (double)P.g.nx * P.g.ny;
    double tot[4] = {0, 0, 0, 0};
    for (int z = 0; z < P.g.nz; ++z) {
        const double* r = &prof[(size_t)z * 5];
        int s = h->zslit[z];
        double n0 = s >= 0 ? (double)h->sl[s].rho0 : 0.0;
        if (n_z) n_z[z] = s >= 0 ? n0 * (1.0 + r[0] / A) : 0.0;
        if (ux_z) ux_z[z] = s >= 0 ? r[1] / A : 0.0;
        if (s < 0) continue;
        tot[0] += n0 * (A + r[0]);
        tot[1] += n0 * r[2];
        tot[2] += n0 * r[3];
        tot[3] += n0 * r[4];
    }
    if (out4)
        for (int k = 0; k < 4; ++k) out4[k] = tot[k];
    return check_status(h);
}

// ||p - q||_2 / (K ||p||_2), max over the two profiles
static double profile_residual(const double* n, const double* n_old, const double* u,
                               const double* u_old, int len, double K)
{
    double worst = 0.0;
    const double* cur[2] = {n, u};
    const double* old[2] = {n_old, u_old};
    for (int k = 0; k < 2; ++k) {
        double dd = 0.0, pp = 0.0;
        for (int z = 0; z < len; ++z) {
            double d = cur[k][z] - old[k][z];
            dd += d * d;
            pp += cur[k][z] * cur[k][z];
        }
        double v = pp > 0 ? sqrt(dd) / (K * sqrt(pp)) : (dd > 0 ? INFINITY : 0.0);
        if (!(v == v)) v = INFINITY;
        worst = fmax(worst, v);
    }
    return worst;
}

extern "C" int lbif_residual(lbif_handle h, double* r, double* mass, double mom[3])
{
    if (!h) return fail(nullptr, LBIF_ERR_ARG, "lbif_residual: NULL handle");
    int nz = h->P.g.nz;
    std::vector<double> n(nz), ux(nz);
    double tot[4];
    int rc = lbif_profiles(h, n.data(), ux.data(), tot);
    double R = INFINITY;
    if (h->last_t >= 0 && h->t > h->last_t)
        R = profile_residual(n.data(), h->last_n.data(), ux.data(), h->last_ux.data(), nz,
                             (double)(h->t - h->last_t));
    h->last_n = n;
    h->last_ux = ux;
    h->last_t = h->t;
    if (r) *r = R;
    if (mass) *mass = tot[0];
    if (mom) {
        mom[0] = tot[1];
        mom[1] = tot[2];
        mom[2] = tot[3];
    }
    return rc;
}

extern "C" int lbif_time(lbif_handle h, int64_t* t)
{
    if (!h || !t) return fail(h, LBIF_ERR_ARG, "lbif_time: bad arguments");
    *t = h->t;
    return LBIF_OK;
}

extern "C" int lbif_status(lbif_handle h, int32_t* status)
{
    if (!h || !status) return fail(h, LBIF_ERR_ARG, "lbif_status: bad arguments");
    int rc = check_status(h);
    *status = h->sticky;
    return rc == LBIF_ERR_DIVERGED ? LBIF_OK : rc;
}

// --------------------------------------------------------------------------
// ensemble
// --------------------------------------------------------------------------
extern "C" int lbif_batch_info(lbif_handle h, int32_t* nslits, int32_t* zlo, int64_t* nodes)
{
    if (!h) return fail(nullptr, LBIF_ERR_ARG, "lbif_batch_info: NULL handle");
    if (nslits) *nslits = (int32_t)h->sl.size();
    if (zlo)
        for (size_t s = 0; s < h->sl.size(); ++s) zlo[s] = h->sl[s].zlo;
    if (nodes) {
        int64_t c = 0;
        for (const SlitParam& s : h->sl) c += (int64_t)(s.zhi - s.zlo + 1) * h->P.g.nx * h->P.g.ny;
        *nodes = c;
    }
    return LBIF_OK;
}

static int upload_done(lbif_ctx* h)
{
    CK(h, cudaMemcpyAsync(h->d_done, h->done.data(), sizeof(int) * h->done.size(),
                          cudaMemcpyHostToDevice, h->stream));
    return LBIF_OK;
}

extern "C" int lbif_batch_seed(lbif_handle h, const float* n_z, const float* ux_z, int32_t hmax)
{
    if (!h || !n_z || hmax < 1) return fail(h, LBIF_ERR_ARG, "lbif_batch_seed: bad arguments");
    for (const SlitParam& s : h->sl)
        if (s.zhi - s.zlo + 1 > hmax) return fail(h, LBIF_ERR_ARG, "lbif_batch_seed: hmax below a slit width");
    size_t cnt = h->sl.size() * (size_t)hmax;
    float* d = nullptr;
    float* tmp = nullptr;  // profiles larger than the scratch (very thin slits): own buffer
    int rc = ensure_scratch(h);
    if (rc) return rc;
    if ((size_t)3 * h->P.g.N >= 2 * cnt) {
        d = h->scratch;
    } else {
        if (cudaMalloc((void**)&tmp, sizeof(float) * 2 * cnt) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, LBIF_ERR_NOMEM, "lbif_batch_seed: device allocation failed");
        }
        d = tmp;
    }
    float* fs[4];
    field_set(h, h->fcur, fs);
    cudaError_t e = cudaMemcpyAsync(d, n_z, sizeof(float) * cnt, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && ux_z)
        e = cudaMemcpyAsync(d + cnt, ux_z, sizeof(float) * cnt, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->pop[h->cur], 0, pop_bytes(h->P) * (size_t)Q * (size_t)h->P.g.Npad, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->clk_d, 0, sizeof(int4) * h->sl.size(), h->stream);
    if (e == cudaSuccess)
        e = launch_init_profiles(h->P, fs, d, ux_z ? d + cnt : nullptr, hmax, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return fail(h, LBIF_ERR_CUDA, std::string("lbif_batch_seed: ") + cudaGetErrorString(e));
    std::fill(h->done.begin(), h->done.end(), 0);
    if ((rc = upload_done(h))) return rc;
    reset_time(h);
    return LBIF_OK;
}

extern "C" int lbif_batch_profiles(lbif_handle h, double* n_z, double* ux_z, int32_t hmax)
{
    if (!h || hmax < 1) return fail(h, LBIF_ERR_ARG, "lbif_batch_profiles: bad arguments");
    std::vector<double> prof;
    int rc = plane_sums(h, prof);
    if (rc) return rc;
    double A = (double)h->P.g.nx * h->P.g.ny;
    for (size_t s = 0; s < h->sl.size(); ++s) {
        const SlitParam& S = h->sl[s];
        for (int j = 0; j < hmax; ++j) {
            int z = S.zlo + j;
            bool in = z <= S.zhi;
            if (n_z) n_z[s * hmax + j] = in ? S.rho0 * (1.0 + prof[(size_t)z * 5] / A) : 0.0;
            if (ux_z) ux_z[s * hmax + j] = in ? prof[(size_t)z * 5 + 1] / A : 0.0;
        }
    }
    return check_status(h);
}

// Host-side buffer indices a captured graph depends on; they repeat with
// period 2 in steady stepping.
static int buffer_state(const lbif_ctx* h) { return h->cur | h->fcur << 1; }

// capture `steps` (even) steps of the active slits into a CUDA graph; the
// graph replays from the buffer state it was captured in, so it is rebuilt
// when that does not hold
static int build_graph(lbif_ctx* h, int steps)
{
    if (h->graph && h->graph_steps == steps && h->graph_state == buffer_state(h)) return LBIF_OK;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    int rc = one_step(h);  // eager step: first-use kernel attributes are set outside capture
    if (rc) return rc;
    rc = one_step(h);
    if (rc) return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    cudaGraph_t g = nullptr;
    const int state = buffer_state(h);
    const int64_t t0 = h->t;
    CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < steps && rc == LBIF_OK; ++k) rc = one_step(h);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    h->t = t0;  // the capture only recorded the launches
    h->G_t = h->tail_t = -1;
    if (rc == LBIF_OK && buffer_state(h) != state)
        rc = fail(h, LBIF_ERR_CUDA, "graph capture: buffer indices do not repeat over the captured steps");
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(h, LBIF_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return fail(h, LBIF_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    h->graph_steps = steps;
    h->graph_state = state;
    return LBIF_OK;
}

// Advance the active slits by `steps` steps through the graph (steps even).
static int run_graph(lbif_ctx* h, int steps)
{
    int rc = build_graph(h, steps);
    if (rc) return rc;
    CK(h, cudaGraphLaunch(h->graph, h->stream));
    h->t += steps;
    invalidate(h);
    return LBIF_OK;
}

extern "C" int lbif_batch_run(lbif_handle h, double tol, int64_t max_steps, int32_t check_every,
                              int32_t patience, int64_t* steps_taken, double* residual)
{
    if (!h || !(tol > 0) || max_steps < 0 || check_every < 2 || patience < 0)
        return fail(h, LBIF_ERR_ARG, "lbif_batch_run: bad arguments");
    const int K = (check_every + 1) / 2 * 2;
    const size_t S = h->sl.size();
    const double A = (double)h->P.g.nx * h->P.g.ny;
    std::fill(h->done.begin(), h->done.end(), 0);
    int rc = upload_done(h);
    if (rc) return rc;
    std::vector<int64_t> taken(S, -1);
    std::vector<double> best(S, INFINITY);
    std::vector<int> since_best(S, 0);
    std::vector<std::vector<double>> pn(S), pu(S);  // previous profiles
    int64_t t0 = h->t;
    size_t active = S;
    std::vector<double> prof;
    while (active > 0 && h->t - t0 < max_steps) {
        if ((rc = run_graph(h, K))) return rc;
        if ((rc = plane_sums(h, prof))) return rc;
        for (size_t s = 0; s < S; ++s) {
            if (h->done[s]) continue;
            const SlitParam& P = h->sl[s];
            int len = P.zhi - P.zlo + 1;
            std::vector<double> n(len), u(len);
            bool bad = false;
            for (int j = 0; j < len; ++j) {
                const double* r = &prof[(size_t)(P.zlo + j) * 5];
                n[j] = P.rho0 * (1.0 + r[0] / A);
                u[j] = r[1] / A;
                bad |= !(n[j] > 0.0) || !isfinite(u[j]);
            }
            if (bad) {
                h->done[s] = 1;  // diverged: frozen, reported as -2
                taken[s] = -2;
                --active;
                continue;
            }
            if (!pn[s].empty()) {
                double R = profile_residual(n.data(), pn[s].data(), u.data(), pu[s].data(), len, (double)K);
                if (R < best[s]) {
                    best[s] = R;
                    since_best[s] = 0;
                } else {
                    ++since_best[s];
                }
                if (R < tol) {
                    h->done[s] = 1;
                    taken[s] = h->t - t0;
                    --active;
                } else if (patience > 0 && since_best[s] >= patience) {
                    h->done[s] = 1;  // rounding floor above tol: frozen, reported as -3
                    taken[s] = -3;
                    --active;
                }
            }
            pn[s].swap(n);
            pu[s].swap(u);
        }
        if ((rc = upload_done(h))) return rc;
    }
    if (steps_taken)
        for (size_t s = 0; s < S; ++s) steps_taken[s] = taken[s];
    if (residual)
        for (size_t s = 0; s < S; ++s) residual[s] = best[s];
    // unfreeze: later calls step every slit again
    std::fill(h->done.begin(), h->done.end(), 0);
    if ((rc = upload_done(h))) return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    return LBIF_OK;
}

extern "C" int lbif_set_fused(lbif_handle h, int32_t fused)
{
    if (!h || (fused != 0 && fused != 1)) return fail(h, LBIF_ERR_ARG, "lbif_set_fused: bad arguments");
    if (!fused)
        return fail(h, LBIF_ERR_UNSUPPORTED,
                    "lbif_set_fused: the two-pass step is retired; populations are stored relative to the "
                    "equilibrium of their own node, which only the pull pass decodes");
    return LBIF_OK;
}

extern "C" int lbif_selftest_wait(int64_t polls, int32_t* timed_out)
{
    if (polls < 1 || !timed_out) return fail(nullptr, LBIF_ERR_ARG, "lbif_selftest_wait: bad arguments");
    int* st = nullptr;
    if (cudaMalloc((void**)&st, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, LBIF_ERR_NOMEM, "lbif_selftest_wait: device allocation failed");
    }
    int v = 0;
    cudaError_t e = cudaMemset(st, 0, sizeof(int));
    if (e == cudaSuccess) e = launch_wait_selftest((long long)polls, st, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(&v, st, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(st);
    if (e != cudaSuccess) return fail(nullptr, LBIF_ERR_CUDA, std::string("lbif_selftest_wait: ") + cudaGetErrorString(e));
    *timed_out = (v & 4) ? 1 : 0;
    return *timed_out ? fail(nullptr, LBIF_ERR_TIMEOUT, "lbif_selftest_wait: the bounded wait ran out")
                      : LBIF_OK;
}

extern "C" int lbif_get_shapes(lbif_handle h, int32_t shapes[5])
{
    if (!h || !shapes) return fail(h, LBIF_ERR_ARG, "lbif_get_shapes: bad arguments");
    shapes[0] = h->ball_want;
    shapes[1] = h->force_group;
    shapes[2] = h->ball_map_ok && h->ball_tma ? 1 : 0;
    shapes[3] = h->csm_lz;
    shapes[4] = h->csm_pf;
    return LBIF_OK;
}

extern "C" int lbif_set_shapes(lbif_handle h, const int32_t shapes[5])
{
    if (!h || !shapes) return fail(h, LBIF_ERR_ARG, "lbif_set_shapes: bad arguments");
    const int32_t* v = shapes;
    if (v[0] < 0 || v[0] > (1 << 20) || v[1] < 0 || v[1] > (1 << 20) || v[2] < 0 || v[2] > 1 || v[3] < 0 ||
        v[3] > (1 << 20) || v[4] < 0 || v[4] > 2)
        return fail(h, LBIF_ERR_ARG, "lbif_set_shapes: value out of range");
    if ((v[2] == 1 && !h->ball_map_ok) || (v[4] == 2 && !h->pop_map_ok))
        return fail(h, LBIF_ERR_UNSUPPORTED, "lbif_set_shapes: this handle has no tensor map for that staging");
    h->ball_want = v[0];
    h->force_group = v[1];
    h->ball_tma = v[2] == 1;
    h->csm_lz = v[3];
    h->csm_pf = v[4];
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return LBIF_OK;
}

extern "C" int lbif_get_fused(lbif_handle h, int32_t* fused)
{
    if (!h || !fused) return fail(h, LBIF_ERR_ARG, "lbif_get_fused: bad arguments");
    *fused = 1;
    return LBIF_OK;
}

// Time each candidate launch shape on the handle's own state and keep the
// fastest: the ball kernel's CTA target (z-chunking) and staging, and the
// force kernel's tile-group edge. The state is saved and restored around the
// trials.
extern "C" int lbif_autotune(lbif_handle h, int32_t trials, int32_t* ball_want, int32_t* force_group,
                             int32_t* ball_staging)
{
    if (!h || trials < 1) return fail(h, LBIF_ERR_ARG, "lbif_autotune: bad arguments");
    const Params& P = h->P;
    int rc = refresh_fields(h, P.hs != 0, 0);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    const int balls[] = {304, 608, 1216, 2432, 4864};
    const int groups[] = {64, 128, 256, 1 << 20};
    float best = 1e30f;
    int best_ball = 0, best_group = 0;
    bool best_tma = h->ball_map_ok;
    float* dnew = h->dn[h->fcur];
    // the ball kernel writes dG only; the force kernel writes F only: both
    // are pure functions of the current fields, so trials change no state.
    // Ball candidates: CTA target x plane staging (tensor-memory-accelerator
    // copies when the handle has tensor maps, plain loads).
    for (int staging = h->ball_map_ok ? 1 : 0; staging >= 0; --staging) {
        const CUtensorMap* tm = staging ? &h->ball_map[h->fcur] : nullptr;
        for (int b : balls) {
            float tot = 0.f;
            for (int k = 0; k < trials + 1; ++k) {
                CK(h, cudaEventRecord(e0, h->stream));
                CK(h, launch_ball(P, dnew, h->dG, h->status_d, b, 0, h->stream, tm));
                CK(h, cudaEventRecord(e1, h->stream));
                CK(h, cudaEventSynchronize(e1));
                float ms;
                CK(h, cudaEventElapsedTime(&ms, e0, e1));
                if (k) tot += ms;
            }
            if (tot < best) {
                best = tot;
                best_ball = b;
                best_tma = staging != 0;
            }
        }
    }
    best = 1e30f;
    for (int gsz : groups) {
        float tot = 0.f;
        for (int k = 0; k < trials + 1; ++k) {
            CK(h, cudaEventRecord(e0, h->stream));
            CK(h, launch_force(P, fields_of(h), h->Ft, h->F, gsz, h->stream));
            CK(h, cudaEventRecord(e1, h->stream));
            CK(h, cudaEventSynchronize(e1));
            float ms;
            CK(h, cudaEventElapsedTime(&ms, e0, e1));
            if (k) tot += ms;
        }
        if (tot < best) {
            best = tot;
            best_group = gsz;
        }
    }
    // Pull pass: z planes per CTA segment x gathers (plain, prefetched one
    // plane ahead, tensor-memory-accelerator boxes when the handle has
    // population maps). A trial reads the
    // current populations and fields and writes only the next step's buffers
    // (not adopted), so trials change no state either.
    int best_lz = h->csm_lz, best_pf = h->csm_pf;
    // (in place a trial would overwrite the state it reads: the pull pass
    // keeps its defaults there)
    if (csm_ok(P.g) && !P.inplace) {
        const float4* Fp = h->F;
        CK(h, launch_force(P, fields_of(h), h->Ft, h->F, best_group, h->stream));
        float* const* u = h->u[h->fcur];
        float* const* w = h->u[h->fcur ^ 1];
        CsmIO io{h->dn[h->fcur], u[0], u[1], u[2], h->dn[h->fcur ^ 1], w[0], w[1], w[2]};
        const int lzs[] = {8, 16, 32};
        best = 1e30f;
        for (int pf = 0; pf <= (h->pop_map_ok ? 2 : 1); ++pf)
            for (int lz : lzs) {
                float tot = 0.f;
                for (int k = 0; k < trials + 1; ++k) {
                    CK(h, cudaEventRecord(e0, h->stream));
                    CK(h, launch_csm(P, h->pop[h->cur], h->pop[h->cur ^ 1], io, Fp, h->status_d, lz, pf, h->stream,
                                     pop_map(h, h->cur)));
                    CK(h, cudaEventRecord(e1, h->stream));
                    CK(h, cudaEventSynchronize(e1));
                    float ms;
                    CK(h, cudaEventElapsedTime(&ms, e0, e1));
                    if (k) tot += ms;
                }
                if (tot < best) {
                    best = tot;
                    best_lz = lz;
                    best_pf = pf;
                }
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->ball_want = best_ball;
    h->force_group = best_group;
    h->ball_tma = best_tma;
    h->csm_lz = best_lz;
    h->csm_pf = best_pf;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    if (ball_want) *ball_want = best_ball;
    if (force_group) *force_group = best_group;
    if (ball_staging) *ball_staging = best_tma ? 1 : 0;
    return check_status(h);
}

// --------------------------------------------------------------------------
// checkpoint: the stored populations and the moment fields they refer to
// (dn, ux, uy, uz); the second population buffer, unused between steps,
// carries the fields between host and device
// --------------------------------------------------------------------------
struct CkptHeader {
    char magic[8];
    int32_t version, nx, ny, nz, sigma, storage;
    int64_t t;
};

static const char kCkptMagic[9] = "LBIFCKP3";

extern "C" int lbif_save(lbif_handle h, const char* path)
{
    if (!h || !path) return fail(h, LBIF_ERR_ARG, "lbif_save: bad arguments");
    const Params& P = h->P;
    int rc = ensure_scratch(h);
    if (rc) return rc;
    size_t es = pop_bytes(P);
    size_t N = (size_t)P.g.N;
    size_t plane = es * N;
    std::vector<char> buf(plane * Q);
    std::vector<float> fld(4 * N);
    // each direction in node order (the layout of the buffer is the
    // library's), then the moment fields
    for (int i = 0; i < Q; ++i) {
        CK(h, launch_pop_canon(P, h->pop[h->cur], i, h->scratch, 0, h->stream));
        CK(h, cudaMemcpyAsync(buf.data() + plane * i, h->scratch, plane, cudaMemcpyDeviceToHost, h->stream));
    }
    float* f[4];
    field_set(h, h->fcur, f);
    CK(h, launch_read_fields(P, f, h->scratch, h->stream));
    CK(h, cudaMemcpyAsync(fld.data(), h->scratch, sizeof(float) * 4 * N, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    FILE* fp = fopen(path, "wb");
    if (!fp) return fail(h, LBIF_ERR_IO, std::string("lbif_save: cannot open ") + path);
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, kCkptMagic, 8);
    hd.version = 3;
    hd.nx = P.g.nx;
    hd.ny = P.g.ny;
    hd.nz = P.g.nz;
    hd.sigma = P.sigma;
    hd.storage = P.storage;
    hd.t = h->t;
    bool ok = fwrite(&hd, sizeof(hd), 1, fp) == 1 && fwrite(buf.data(), 1, buf.size(), fp) == buf.size() &&
              fwrite(fld.data(), sizeof(float), 4 * N, fp) == 4 * N;
    ok = (fclose(fp) == 0) && ok;
    return ok ? LBIF_OK : fail(h, LBIF_ERR_IO, "lbif_save: write failed");
}

extern "C" int lbif_load(lbif_handle h, const char* path)
{
    if (!h || !path) return fail(h, LBIF_ERR_ARG, "lbif_load: bad arguments");
    const Params& P = h->P;
    int rc = ensure_scratch(h);
    if (rc) return rc;
    FILE* fp = fopen(path, "rb");
    if (!fp) return fail(h, LBIF_ERR_IO, std::string("lbif_load: cannot open ") + path);
    CkptHeader hd;
    size_t es = pop_bytes(P);
    size_t N = (size_t)P.g.N;
    size_t plane = es * N;
    std::vector<char> buf(plane * Q);
    std::vector<float> fld(4 * N);
    bool ok = fread(&hd, sizeof(hd), 1, fp) == 1 && memcmp(hd.magic, kCkptMagic, 8) == 0 &&
              hd.nx == P.g.nx && hd.ny == P.g.ny && hd.nz == P.g.nz && hd.sigma == P.sigma &&
              hd.storage == P.storage && fread(buf.data(), 1, buf.size(), fp) == buf.size() &&
              fread(fld.data(), sizeof(float), 4 * N, fp) == 4 * N;
    fclose(fp);
    if (!ok) return fail(h, LBIF_ERR_IO, "lbif_load: file does not match this handle");
    if ((rc = zero_populations(h))) return rc;  // the clocks restart: node-order slots
    for (int i = 0; i < Q; ++i) {
        CK(h, cudaMemcpyAsync(h->scratch, buf.data() + plane * i, plane, cudaMemcpyHostToDevice, h->stream));
        CK(h, launch_pop_canon(P, h->pop[h->cur], i, h->scratch, 1, h->stream));
    }
    float* f[4];
    field_set(h, h->fcur, f);
    CK(h, cudaMemcpyAsync(h->scratch, fld.data(), sizeof(float) * 4 * N, cudaMemcpyHostToDevice, h->stream));
    CK(h, launch_write_fields(P, h->scratch, f, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    reset_time(h);
    h->t = hd.t;
    return LBIF_OK;
}
