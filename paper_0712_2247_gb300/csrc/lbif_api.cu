// Host side of the C ABI declared in include/lbif.h: argument checks, the
// quadrature / ball / tail tables (built in FP64, rounded once to FP32),
// device allocation and the per-step launch sequence.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "lbif_internal.h"

using namespace lbif;

struct lbif_ctx {
    Params P;
    cudaStream_t stream = nullptr;
    void* pop[2] = {nullptr, nullptr};
    int cur = 0;                      // populations of the current step
    float* dn[2] = {nullptr, nullptr};
    int dcur = 0;                     // dn[dcur] = reference of pop[cur]
    float* ux = nullptr;
    float* uy = nullptr;
    float* uz = nullptr;
    float* dG = nullptr;
    float4* Ft = nullptr;
    float4* F = nullptr;              // F / n0 per node (force kernel -> collision kernel)
    int* tail_off = nullptr;
    float4* tail_K = nullptr;
    int tail_pairs = 0;
    int* status_d = nullptr;
    double* prof_d = nullptr;
    float* scratch = nullptr;         // 3 N floats, for host-side outputs
    int64_t t = 0;
    int64_t fields_t = -1, G_t = -1, tail_t = -1;  // step the cached fields belong to
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

// padded fields carry PAD_SLACK floats before their first element
static float* padded_alloc(size_t P)
{
    float* raw = nullptr;
    if (cudaMalloc((void**)&raw, sizeof(float) * (P + 2 * PAD_SLACK)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return raw + PAD_SLACK;
}

static void padded_free(float* p)
{
    if (p) cudaFree(p - PAD_SLACK);
}

static void free_ctx(lbif_ctx* h)
{
    if (!h) return;
    void* bufs[] = {h->pop[0], h->pop[1], h->Ft,     h->F,      h->tail_off,
                    h->tail_K, h->status_d, h->prof_d, h->scratch};
    for (void* b : bufs)
        if (b) cudaFree(b);
    float* pads[] = {h->dn[0], h->dn[1], h->ux, h->uy, h->uz, h->dG};
    for (float* q : pads) padded_free(q);
    delete h;
}

static Fields fields_of(const lbif_ctx* h)
{
    Fields f;
    f.dn = h->dn[h->dcur ^ 1];
    f.ux = h->ux;
    f.uy = h->uy;
    f.uz = h->uz;
    f.dG = h->dG;
    return f;
}

static void invalidate(lbif_ctx* h) { h->fields_t = h->G_t = h->tail_t = -1; }

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

// --------------------------------------------------------------------------
// create / destroy
// --------------------------------------------------------------------------
extern "C" int lbif_create(lbif_handle* out, lbif_grid gr, double sigma, double eta, double tau,
                           lbif_walls w, const lbif_force* f, const lbif_opts* o)
{
    if (!out) return fail(nullptr, LBIF_ERR_ARG, "lbif_create: out is NULL");
    *out = nullptr;
    if (gr.nx < 1 || gr.ny < 1 || gr.nz < 1)
        return fail(nullptr, LBIF_ERR_ARG, "lbif_create: grid extents must be >= 1");
    if (!(sigma >= 2.0) || sigma != floor(sigma) || ((int)sigma) % 2 != 0 || sigma > MAX_SIGMA)
        return fail(nullptr, LBIF_ERR_UNSUPPORTED,
                    "lbif_create: sigma must be an even integer in [2, 24] lattice spacings");
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
    if (O.storage != LBIF_STORE_F32 && O.storage != LBIF_STORE_F16)
        return fail(nullptr, LBIF_ERR_ARG, "lbif_create: storage must be 0 (FP32) or 1 (FP16)");
    if (!(O.noise >= 0.0 && O.noise < 1.0)) return fail(nullptr, LBIF_ERR_ARG, "lbif_create: noise must be in [0,1)");
    if (F.tail && !(F.rcut >= 1.0 && F.rcut <= 4.0 && F.eps >= 0.0))
        return fail(nullptr, LBIF_ERR_ARG, "lbif_create: tail needs rcut in [1,4] and eps >= 0");
    if ((F.g2_form != 0 && F.g2_form != 1))
        return fail(nullptr, LBIF_ERR_ARG, "lbif_create: g2_form must be 0 or 1");
    for (int a = 0; a < 3; ++a)
        if (!isfinite(F.body[a])) return fail(nullptr, LBIF_ERR_ARG, "lbif_create: body force not finite");

    lbif_ctx* h = new lbif_ctx();
    memset(&h->P, 0, sizeof(Params));
    Params& P = h->P;
    int s = (int)sigma;
    Geom& g = P.g;
    g.nx = gr.nx;
    g.ny = gr.ny;
    g.nz = gr.nz;
    g.zper = (w.z == LBIF_PERIODIC);
    g.hw = s;
    if (F.tail) g.hw = std::max(g.hw, (int)ceil(F.rcut * s));
    g.hw = (g.hw + 3) / 4 * 4;                   // rows 16-byte aligned
    g.px = (g.nx + 2 * g.hw + 8 + 3) / 4 * 4;    // + slack columns for float4 windows
    g.py = g.ny + 2 * g.hw;
    g.pz = g.nz + 2 * g.hw;
    g.N = (long long)g.nx * g.ny * g.nz;
    g.Npad = (g.N + 63) / 64 * 64;
    g.P = (long long)g.px * g.py * g.pz;
    if (g.P >= (1LL << 31)) {
        delete h;
        return fail(nullptr, LBIF_ERR_UNSUPPORTED, "lbif_create: padded grid exceeds 2^31 nodes");
    }
    const double kT = 1.0 / 3.0;
    double n0 = 6.0 * eta / (M_PI * sigma * sigma * sigma);
    P.sigma = s;
    P.inv_tau = (float)(1.0 / tau);
    P.rho0 = (float)n0;
    P.eta0 = (float)eta;
    P.G0 = (float)g2_host(eta, F.g2_form);
    P.hs_pref = (float)(-kT * sigma * sigma * 4.0 * M_PI * n0);
    P.p_pref = (float)(kT * sigma * sigma * sigma / 6.0 * 4.0 * M_PI * n0 * n0);
    P.kappa = (float)(2.0 / (sqrt(kT) * sqrt(M_PI)));
    P.inv_sigma = (float)(1.0 / sigma);
    P.ball_inv = (float)(1.0 / ball_count(s));
    for (int a = 0; a < 3; ++a) P.body[a] = (float)F.body[a];
    P.hs = F.hs ? 1 : 0;
    P.coupling = F.coupling ? 1 : 0;
    P.regularize = F.regularize ? 1 : 0;
    P.g2form = F.g2_form;
    P.tail = F.tail ? 1 : 0;
    P.storage = O.storage;
    {
        const int cx[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        const int cy[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        const int cz[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        for (int i = 0; i < Q; ++i) {
            P.nbr[i] = padded_offset(g, cx[i], cy[i], cz[i]);
            P.soff[i] = cx[i] + (long long)cy[i] * g.nx + (long long)cz[i] * g.nx * g.ny;
        }
    }
    if (build_shell(P)) {
        delete h;
        return fail(nullptr, LBIF_ERR_UNSUPPORTED, "lbif_create: quadrature tables do not fit");
    }
    h->stream = (cudaStream_t)O.stream;

    // tail taps: one representative of each +-d pair with sigma <= |d| <= rcut sigma
    std::vector<int> toff;
    std::vector<float4> tK;
    if (P.tail) {
        double rmax = F.rcut * sigma;
        int R = (int)ceil(rmax);
        double s6 = pow(sigma, 6.0), s12 = s6 * s6;
        for (int dz = 0; dz <= R; ++dz)
            for (int dy = (dz == 0 ? 0 : -R); dy <= R; ++dy)
                for (int dx = ((dz == 0 && dy == 0) ? 1 : -R); dx <= R; ++dx) {
                    double r2 = (double)dx * dx + (double)dy * dy + (double)dz * dz;
                    if (r2 < sigma * sigma || r2 > rmax * rmax) continue;
                    double r = sqrt(r2);
                    double dphi = 4.0 * F.eps * (-12.0 * s12 / pow(r, 13.0) + 6.0 * s6 / pow(r, 7.0));
                    toff.push_back(padded_offset(g, dx, dy, dz));
                    tK.push_back(make_float4((float)(dphi * dx / r), (float)(dphi * dy / r),
                                             (float)(dphi * dz / r), 0.f));
                }
        h->tail_pairs = (int)toff.size();
    }

    size_t pb = pop_bytes(P) * (size_t)Q * (size_t)g.Npad;
#define ALLOC(ptr, bytes)                                                                   \
    do {                                                                                    \
        if (cudaMalloc((void**)&(ptr), (bytes)) != cudaSuccess) {                           \
            cudaGetLastError();                                                             \
            free_ctx(h);                                                                    \
            return fail(nullptr, LBIF_ERR_NOMEM, "lbif_create: device allocation failed");  \
        }                                                                                   \
    } while (0)
    ALLOC(h->pop[0], pb);
    ALLOC(h->pop[1], pb);
    ALLOC(h->F, sizeof(float4) * (size_t)g.N);
    ALLOC(h->status_d, sizeof(int));
    ALLOC(h->prof_d, sizeof(double) * 5 * (size_t)g.nz);
    if (P.tail) {
        ALLOC(h->Ft, sizeof(float4) * (size_t)g.N);
        ALLOC(h->tail_off, sizeof(int) * toff.size());
        ALLOC(h->tail_K, sizeof(float4) * tK.size());
    }
    {
        float** pads[] = {&h->dn[0], &h->dn[1], &h->ux, &h->uy, &h->uz, &h->dG};
        for (float** q : pads) {
            *q = padded_alloc((size_t)g.P);
            if (!*q) {
                free_ctx(h);
                return fail(nullptr, LBIF_ERR_NOMEM, "lbif_create: device allocation failed");
            }
        }
    }
#undef ALLOC
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
    CKC(cudaMemsetAsync(h->pop[0], 0, pb, h->stream));
    CKC(cudaMemsetAsync(h->pop[1], 0, pb, h->stream));
    {
        float* pads[] = {h->dn[0], h->dn[1], h->ux, h->uy, h->uz, h->dG};
        const float outside[] = {-1.f, -1.f, 0.f, 0.f, 0.f, 0.f};
        for (float* q : pads)
            CKC(cudaMemsetAsync(q - PAD_SLACK, 0, sizeof(float) * ((size_t)g.P + 2 * PAD_SLACK), h->stream));
        CKC(launch_fill_outside(P, pads, outside, 6, h->stream));
    }
    CKC(cudaMemsetAsync(h->status_d, 0, sizeof(int), h->stream));
    if (P.tail) {
        CKC(cudaMemcpyAsync(h->tail_off, toff.data(), sizeof(int) * toff.size(),
                            cudaMemcpyHostToDevice, h->stream));
        CKC(cudaMemcpyAsync(h->tail_K, tK.data(), sizeof(float4) * tK.size(),
                            cudaMemcpyHostToDevice, h->stream));
    }
    CKC(launch_init_noise(P, h->pop[0], h->dn[0], O.seed, O.noise, 0, h->stream));
    CKC(cudaStreamSynchronize(h->stream));
#undef CKC
    *out = h;
    return LBIF_OK;
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
// Moments (and, when asked, the g2 field and the tail force) of the current
// populations; cached per step so that output calls between steps do not
// redo them. The new dn goes to dn[dcur^1]; the reference dn[dcur] is kept.
static int refresh_fields(lbif_ctx* h, bool want_G)
{
    const Params& P = h->P;
    float* dnew = h->dn[h->dcur ^ 1];
    if (h->fields_t != h->t) {
        CK(h, launch_moments(P, h->pop[h->cur], h->dn[h->dcur], dnew, h->ux, h->uy, h->uz,
                             h->status_d, h->stream));
        h->fields_t = h->t;
    }
    if (want_G && h->G_t != h->t) {
        CK(h, launch_ball(P, dnew, h->dG, h->status_d, h->stream));
        h->G_t = h->t;
    }
    if (P.tail && h->tail_t != h->t) {
        CK(h, launch_tail(P, dnew, h->tail_off, h->tail_K, h->tail_pairs, h->Ft, h->stream));
        h->tail_t = h->t;
    }
    return LBIF_OK;
}

static int advance(lbif_ctx* h)
{
    const Params& P = h->P;
    const Fields f = fields_of(h);
    CK(h, launch_force(P, f, h->Ft, h->F, h->stream));
    CK(h, launch_cs(P, h->pop[h->cur], h->pop[h->cur ^ 1], f, h->F, h->stream));
    h->cur ^= 1;
    h->dcur ^= 1;
    h->t += 1;
    return LBIF_OK;
}

extern "C" int lbif_step(lbif_handle h, int64_t nsteps)
{
    if (!h || nsteps < 0) return fail(h, LBIF_ERR_ARG, "lbif_step: bad arguments");
    for (int64_t k = 0; k < nsteps; ++k) {
        int rc = refresh_fields(h, h->P.hs != 0);
        if (rc) return rc;
        if ((rc = advance(h))) return rc;
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
    int per = 3 + (P.hs ? 1 : 0) + (P.tail ? 1 : 0);
    std::vector<cudaEvent_t> ev((size_t)nsteps * per + 1);
    std::vector<int> cls((size_t)nsteps * per);
    for (auto& e : ev) CK(h, cudaEventCreate(&e));
    size_t j = 0;
    CK(h, cudaEventRecord(ev[0], h->stream));
    for (int64_t s = 0; s < nsteps; ++s) {
        float* dnew = h->dn[h->dcur ^ 1];
        const Fields f = fields_of(h);
        CK(h, launch_moments(P, h->pop[h->cur], h->dn[h->dcur], dnew, h->ux, h->uy, h->uz,
                             h->status_d, h->stream));
        cls[j] = 0;
        CK(h, cudaEventRecord(ev[++j], h->stream));
        if (P.hs) {
            CK(h, launch_ball(P, dnew, h->dG, h->status_d, h->stream));
            cls[j] = 1;
            CK(h, cudaEventRecord(ev[++j], h->stream));
        }
        if (P.tail) {
            CK(h, launch_tail(P, dnew, h->tail_off, h->tail_K, h->tail_pairs, h->Ft, h->stream));
            cls[j] = 2;
            CK(h, cudaEventRecord(ev[++j], h->stream));
        }
        CK(h, launch_force(P, f, h->Ft, h->F, h->stream));
        cls[j] = 3;
        CK(h, cudaEventRecord(ev[++j], h->stream));
        CK(h, launch_cs(P, h->pop[h->cur], h->pop[h->cur ^ 1], f, h->F, h->stream));
        cls[j] = 4;
        CK(h, cudaEventRecord(ev[++j], h->stream));
        h->cur ^= 1;
        h->dcur ^= 1;
        h->t += 1;
    }
    invalidate(h);
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
    if (h->sticky)
        return fail(h, LBIF_ERR_DIVERGED,
                    (h->sticky & 2) ? "state diverged: coarse-grained packing fraction reached 1"
                                    : "state diverged: non-finite or non-positive density");
    return LBIF_OK;
}

static int ensure_scratch(lbif_ctx* h)
{
    if (h->scratch) return LBIF_OK;
    if (cudaMalloc((void**)&h->scratch, sizeof(float) * 3 * (size_t)h->P.g.N) != cudaSuccess) {
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
    int rc = refresh_fields(h, pressure && P.hs);
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
    int rc = refresh_fields(h, P.hs != 0);
    if (rc) return rc;
    // the same force kernel as the time step, then a layout change to SoA
    CK(h, launch_force(P, fields_of(h), h->Ft, h->F, h->stream));
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
        // rho goes to the (not yet used) second population buffer, u to the scratch
        float* d = (float*)h->pop[h->cur ^ 1];
        CK(h, cudaMemcpyAsync(d, rho, sizeof(float) * N, cudaMemcpyHostToDevice, h->stream));
        drho = d;
        if (u) {
            CK(h, cudaMemcpyAsync(h->scratch, u, sizeof(float) * 3 * N, cudaMemcpyHostToDevice,
                                  h->stream));
            du = h->scratch;
        }
    }
    CK(h, launch_init_fields(P, h->pop[h->cur], h->dn[h->dcur], drho, du, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->t = 0;
    h->last_t = -1;
    invalidate(h);
    return LBIF_OK;
}

extern "C" int lbif_profiles(lbif_handle h, double* n_z, double* ux_z, double* out4)
{
    if (!h) return fail(nullptr, LBIF_ERR_ARG, "lbif_profiles: NULL handle");
    const Params& P = h->P;
    int nz = P.g.nz;
    int rc = refresh_fields(h, false);
    if (rc) return rc;
    CK(h, launch_profiles(P, fields_of(h), h->prof_d, h->stream));
    std::vector<double> prof((size_t)nz * 5);
    CK(h, cudaMemcpyAsync(prof.data(), h->prof_d, sizeof(double) * prof.size(),
                          cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    double A = (double)P.g.nx * P.g.ny;
    double n0 = (double)P.rho0;
    double tot[4] = {0, 0, 0, 0};
    for (int z = 0; z < nz; ++z) {
        const double* r = &prof[(size_t)z * 5];
        if (n_z) n_z[z] = n0 * (1.0 + r[0] / A);
        if (ux_z) ux_z[z] = r[1] / A;
        tot[0] += A + r[0];
        tot[1] += r[2];
        tot[2] += r[3];
        tot[3] += r[4];
    }
    if (out4)
        for (int k = 0; k < 4; ++k) out4[k] = n0 * tot[k];
    return check_status(h);
}

extern "C" int lbif_residual(lbif_handle h, double* r, double* mass, double mom[3])
{
    if (!h) return fail(nullptr, LBIF_ERR_ARG, "lbif_residual: NULL handle");
    int nz = h->P.g.nz;
    std::vector<double> n(nz), ux(nz);
    double tot[4];
    int rc = lbif_profiles(h, n.data(), ux.data(), tot);
    double R = INFINITY;
    if (h->last_t >= 0 && h->t > h->last_t) {
        double K = (double)(h->t - h->last_t);
        double worst = 0.0;
        const std::vector<double>* cur[2] = {&n, &ux};
        const std::vector<double>* old[2] = {&h->last_n, &h->last_ux};
        for (int k = 0; k < 2; ++k) {
            double dd = 0.0, pp = 0.0;
            for (int z = 0; z < nz; ++z) {
                double d = (*cur[k])[z] - (*old[k])[z];
                dd += d * d;
                pp += (*cur[k])[z] * (*cur[k])[z];
            }
            double v = pp > 0 ? sqrt(dd) / (K * sqrt(pp)) : (dd > 0 ? INFINITY : 0.0);
            worst = fmax(worst, v);
        }
        R = worst;
    }
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
// checkpoint: populations and their reference density field
// --------------------------------------------------------------------------
struct CkptHeader {
    char magic[8];
    int32_t version, nx, ny, nz, sigma, storage;
    int64_t t;
};

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
    std::vector<float> ref(N);
    for (int i = 0; i < Q; ++i)
        CK(h, cudaMemcpyAsync(buf.data() + plane * i, (char*)h->pop[h->cur] + es * (size_t)P.g.Npad * i,
                              plane, cudaMemcpyDeviceToHost, h->stream));
    CK(h, launch_read_ref(P, h->dn[h->dcur], h->scratch, h->stream));
    CK(h, cudaMemcpyAsync(ref.data(), h->scratch, sizeof(float) * N, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    FILE* fp = fopen(path, "wb");
    if (!fp) return fail(h, LBIF_ERR_IO, std::string("lbif_save: cannot open ") + path);
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "LBIFCKP2", 8);
    hd.version = 2;
    hd.nx = P.g.nx;
    hd.ny = P.g.ny;
    hd.nz = P.g.nz;
    hd.sigma = P.sigma;
    hd.storage = P.storage;
    hd.t = h->t;
    bool ok = fwrite(&hd, sizeof(hd), 1, fp) == 1 && fwrite(buf.data(), 1, buf.size(), fp) == buf.size() &&
              fwrite(ref.data(), sizeof(float), N, fp) == N;
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
    std::vector<float> ref(N);
    bool ok = fread(&hd, sizeof(hd), 1, fp) == 1 && memcmp(hd.magic, "LBIFCKP2", 8) == 0 &&
              hd.nx == P.g.nx && hd.ny == P.g.ny && hd.nz == P.g.nz && hd.sigma == P.sigma &&
              hd.storage == P.storage && fread(buf.data(), 1, buf.size(), fp) == buf.size() &&
              fread(ref.data(), sizeof(float), N, fp) == N;
    fclose(fp);
    if (!ok) return fail(h, LBIF_ERR_IO, "lbif_load: file does not match this handle");
    for (int i = 0; i < Q; ++i)
        CK(h, cudaMemcpyAsync((char*)h->pop[h->cur] + es * (size_t)P.g.Npad * i, buf.data() + plane * i,
                              plane, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->scratch, ref.data(), sizeof(float) * N, cudaMemcpyHostToDevice, h->stream));
    CK(h, launch_write_ref(P, h->scratch, h->dn[h->dcur], h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->t = hd.t;
    h->last_t = -1;
    invalidate(h);
    return LBIF_OK;
}
