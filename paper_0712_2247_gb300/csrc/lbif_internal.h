// Internal definitions shared by the host API and the device kernels.
//
// State of a slit on the device:
//   pop[2]  19 planes of Npad elements (FP32 or FP16), node index
//           idx = (z*ny + y)*nx + x, two buffers, pull streaming; or, in
//           place, one buffer in which direction i of a node moves by c_i
//           slots every step (see the pull pass). A population
//           is stored as its non-equilibrium part relative to the node's own
//           equilibrium weight, h_i = s (f_i - f_i^eq(n, u)) / (w_i n), at the
//           moments n, u of the step it belongs to (s = 2^8 for FP16, 1 for
//           FP32); the equilibrium part is carried by those moments.
//   dn[2], u[2][3]  the moments of that step and of the next one (written by
//           the pull pass): dn = n/n0 - 1 and u = j/n, float on a padded grid
//           (halo hw on every side).
//   dG      float  g2(etabar) - g2(eta0) on the padded grid.
//   F       float4 F/n0 per node (force kernel -> collision kernel).
//   The x/y halo holds periodic images written by the producing kernel; the
//   z halo holds images (periodic z) or the constant outside-the-fluid values
//   dn = -1, u = 0, dG = 0 (slit), so stencils need no bounds tests. Padded
//   rows are 16-byte aligned (hw and px multiples of 4) so four consecutive x
//   nodes are one float4; every padded array has 64 floats of slack on both
//   sides for the vector windows of the stencils.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbif.h"

namespace lbif {

constexpr int Q = 19;
constexpr int MAX_SIGMA = 24;
constexpr int PAD_SLACK = 64;  // floats before and after every padded array

struct Geom {
    int nx, ny, nz;
    int hw;          // halo width of the padded fields (multiple of 4)
    int px, py, pz;  // padded extents (px multiple of 4)
    int zper;
    long long N;     // nx*ny*nz
    long long Npad;  // population plane stride (N rounded up to 64)
    long long P;     // px*py*pz
};

// 18-point sphere rule, stencils as padded-grid offsets.
//   axis pair a (a = x, y, z): neighbour at +-sigma e_a, midpoint at +-sigma/2 e_a
//   face-diagonal quartet of plane (a, b) = (x,y), (x,z), (y,z): the four
//     points sigma (sa e_a + sb e_b)/sqrt2, sa, sb = +-1. Each interpolates its
//     neighbour (and midpoint) from the corners (sa (lo + ka), sb (lo + kb)),
//     ka, kb in {0, 1}, with the weights w[k], k = ka + 2 kb, shared by all
//     four members in the same order, so mirror images sum bit-identically.
//     nb_a[k] = (lo + ka) * stride_a, nb_b[k] = (lo + kb) * stride_b.
struct Shell {
    int ax_nb[3];
    int ax_md[3];
    int nb_a[3][4], nb_b[3][4];
    float nb_w[3][4];
    int md_a[3][4], md_b[3][4];
    float md_w[3][4];
};

// Per-slit parameters. A handle holds one slit (z planes 0..nz-1) or an
// ensemble of slits stacked along z with hw planes of "outside" between them;
// zslit[z] gives the slit of a plane (-1 for a gap plane).
struct SlitParam {
    float rho0;      // n0 of the slit
    float eta0;
    float G0;        // g2(eta0)
    float inv_tau;
    float hs_pref;   // -kT sigma^2 4 pi n0
    float p_pref;    // kT sigma^3/6 4 pi n0^2
    float body[3];   // F_e per particle
    int zlo, zhi;    // first and last fluid plane
    int zb, R;       // in place: the slit's ring of R storage planes starts at plane zb
};

struct Params {
    Geom g;
    float kappa;     // 2/(v_T sqrt(pi))
    float inv_sigma;
    float ball_inv;  // 1 / ball node count
    int sigma;
    int hs, coupling, regularize, g2form, tail, storage;
    int c2;               // energy source of Eq. C2eq on (F.w carries C2 / n0)
    int shifted;          // velocity-shifted second-order forcing (equilibrium at u + F/(2n))
    int nslits;
    const SlitParam* sl;  // device table, nslits entries
    const int* zslit;     // device table, nz entries
    const int* done;      // device flags, nslits entries (1 = frozen)
    int inplace;          // populations in one buffer (shifting slots)
    const int4* clk;      // in place: per slit (t mod nx, t mod ny, t mod R) of its step t
    int nbr[Q];           // padded offsets of the 19 lattice neighbours
    long long soff[Q];    // node-index offsets of the 19 neighbours (no wrap)
    long long dbase[Q];   // i Npad: start of direction i in a population buffer
    long long doff[Q];    // i Npad - soff[i]: where node idx pulls direction i from (no wrap)
    unsigned dbase32[Q];  // in place: i Npad (the layout keeps Q Npad below 2^32)
    Shell sh;
};

// moment fields of the current step (padded)
struct Fields {
    const float* dn;
    const float* ux;
    const float* uy;
    const float* uz;
    const float* dG;
};

// inputs and outputs of the pull pass (padded fields; the outputs are other
// buffers than the inputs)
struct CsmIO {
    const float* dn;    // dn(t), the moments the stored populations refer to
    const float* ux;
    const float* uy;
    const float* uz;    // u(t)
    float* dnw;         // dn(t + 1), the moments of the new populations
    float* uxw;
    float* uyw;
    float* uzw;         // u(t + 1)
};

// ---- launchers (lbif_kernels.cu) -------------------------------------------
cudaError_t launch_fill_outside(const Params& P, float* const* planes, const float* values,
                                int nplanes, cudaStream_t s);
// the initial states are equilibria: the caller zeroes the stored populations
cudaError_t launch_init_noise(const Params& P, float* dn, uint64_t seed, double amp, long long offset,
                              cudaStream_t s);
// f[4]: the padded fields dn, ux, uy, uz of the state being set
cudaError_t launch_init_profiles(const Params& P, float* const f[4], const float* n_z, const float* ux_z,
                                 int hmax, cudaStream_t s);
cudaError_t launch_init_fields(const Params& P, float* const f[4], const float* rho, const float* u,
                               cudaStream_t s);
// in place: advance the clocks of the slits not frozen (after every pull pass)
cudaError_t launch_tick(const Params& P, int4* clk, cudaStream_t s);
// the populations of direction i of the current state in node order (N
// elements; gap planes skipped) <-> the buffer (to_pop: scatter into it)
cudaError_t launch_pop_canon(const Params& P, void* pop, int i, void* canon, int to_pop, cudaStream_t s);
// the four fields <-> four unpadded N-arrays (checkpoints)
cudaError_t launch_write_fields(const Params& P, const float* src, float* const f[4], cudaStream_t s);
cudaError_t launch_read_fields(const Params& P, const float* const f[4], float* out, cudaStream_t s);
// want: CTAs to aim for when splitting z into chunks (<= 0: default).
// tmap: a 3-D tensor map of dn (padded extents px, py, pz; box from
// ball_box) to stage the plane tiles with the tensor-memory accelerator, or
// NULL for plain loads. Bit 4 of status records a bounded wait that ran out.
cudaError_t launch_ball(const Params& P, const float* dn, float* dG, int* status, int want,
                        int skip_done, cudaStream_t s, const CUtensorMap* tmap = nullptr);
// box (x extent W, y extent H) of the ball kernel's plane tile for sigma
void ball_box(int sigma, int* W, int* H);
cudaError_t launch_tail(const Params& P, const float* dn, const int* off, const float4* K,
                        int npairs, float4* Ft, cudaStream_t s);
// group: edge (nodes) of the x-y block the resident CTAs sweep together (<= 0: default)
cudaError_t launch_force(const Params& P, const Fields& f, const float4* Ft, float4* F, int group,
                         cudaStream_t s);
// ---- spectral tail (lbif_fft.cu) -------------------------------------------
// usable when nx and ny are powers of two in [2, 1024] and nx ny >= 32
bool tail_spectral_ok(const Geom& g);
// bytes of the work buffer for a kernel reaching D planes in z
size_t tail_spectral_bytes(const Geom& g, int D);
// transform the tail kernel (pairs +-d with displacements pdx, pdy, pdz and
// vector weights K) into the work buffer; synchronises s
cudaError_t tail_spectral_init(const Geom& g, int D, const int* pdx, const int* pdy, const int* pdz,
                               const float4* K, int npairs, const int* zslit, float2* work, cudaStream_t s);
// Ft = the tail force / n0 from the density deviation field dn (padded)
cudaError_t launch_tail_spectral(const Params& P, const float* dn, int D, float2* work, float4* Ft,
                                 cudaStream_t s);
// one step's collision, pull streaming and the moments of the new
// populations (CsmIO); lz: z planes per CTA segment of the tiled kernel
// (<= 0: default); prefetch: 0 plain, 1 the next plane's population gathers
// issued before the current plane is collided, 2 the gathers brought in by
// the tensor-memory accelerator from pmap (a 4-D map of pin: x, y, z,
// direction, box from pop_box; two-buffer layout only; bit 4 of status
// records a bounded wait that ran out). Grids narrower than one tile run the
// per-node kernel (lz, prefetch unused).
bool csm_ok(const Geom& g);
cudaError_t launch_csm(const Params& P, const void* pin, void* pout, const CsmIO& io, const float4* F,
                       int* status, int lz, int prefetch, cudaStream_t s, const CUtensorMap* pmap = nullptr);
// box (x extent W, y extent H) of the tensor-memory-accelerator pull pass
void pop_box(int storage, int* W, int* H);
// bounded mbarrier wait on a barrier nothing completes: sets bit 4 of status
cudaError_t launch_wait_selftest(long long polls, int* status, cudaStream_t s);
cudaError_t launch_force_soa(const Params& P, const float4* F, float* out, cudaStream_t s);
cudaError_t launch_moments_out(const Params& P, const Fields& f, float* rho, float* u, float* p,
                               cudaStream_t s);
// prof: at least profile_doubles(g) doubles; the first 5 nz receive the
// per-plane sums (dn, ux, (1+dn) ux, (1+dn) uy, (1+dn) uz), the rest is work space
size_t profile_doubles(const Geom& g);
cudaError_t launch_profiles(const Params& P, const Fields& f, double* prof, cudaStream_t s);
bool force_vectorised(int sigma);

}  // namespace lbif
