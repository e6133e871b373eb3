// Internal definitions shared by the host API and the device kernels.
//
// Device data layout (one slit):
//   pop[2]  19 planes of Npad elements (FP32 or FP16), h_i = f_i/(w_i n0) - 1,
//           node index idx = (z*ny + y)*nx + x; two buffers, push streaming.
//   M       float4 {dn, ux, uy, uz} on a padded grid (halo hw on every side):
//           dn = n/n0 - 1 (relative density deviation), u = j/n.
//   dn      float  dn on the same padded grid (ball sums read this).
//   dG      float  g2(etabar) - g2(eta0) on the padded grid.
//   The x/y halo holds periodic images written by the producing kernel; the
//   z halo holds images (periodic z) or the constant outside-the-fluid values
//   dn = -1, u = 0, dG = 0 (slit), so stencils need no bounds tests.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbif.h"

namespace lbif {

constexpr int Q = 19;
constexpr int NSHELL = 18;
constexpr int MAX_SEG = 192;  // ball row segments (113 at sigma = 12)
constexpr int MAX_SIGMA = 24;

struct Geom {
    int nx, ny, nz;
    int hw;          // halo width of the padded fields
    int px, py, pz;  // padded extents
    int zper;
    long long N;     // nx*ny*nz
    long long Npad;  // population plane stride (N rounded up to 64)
    long long P;     // px*py*pz
};

// One point of the 18-point sphere rule with its interpolation stencils,
// already converted to padded-grid offsets.
struct ShellPoint {
    float dir[3];
    float w;
    int nnb;         // 1 (on-lattice) or 4 (bilinear) neighbour corners
    int nmd;         // same for the midpoint
    int nb_off[4];
    float nb_w[4];
    int md_off[4];
    float md_w[4];
};

struct Params {
    Geom g;
    float inv_tau;
    float rho0;      // n0
    float eta0;
    float G0;        // g2(eta0)
    float hs_pref;   // -kT sigma^2 4 pi n0
    float p_pref;    // kT sigma^3/6 4 pi n0^2
    float kappa;     // 2/(v_T sqrt(pi))
    float inv_sigma;
    float ball_inv;  // 1 / ball node count
    float body[3];
    int sigma;
    int hs, coupling, regularize, g2form, tail, storage;
    int nseg;
    int seg_off[MAX_SEG];  // padded offset of the first node of each row
    int seg_len[MAX_SEG];
    ShellPoint sp[NSHELL];  // antipodal pairs at (2k, 2k+1)
};

// ---- launchers (lbif_kernels.cu) -------------------------------------------
cudaError_t launch_fill_outside(const Params& P, float4* M, float* dn, float* dG, cudaStream_t s);
cudaError_t launch_init_noise(const Params& P, void* pop, uint64_t seed, double amp,
                              long long offset, cudaStream_t s);
cudaError_t launch_init_fields(const Params& P, void* pop, const float* rho, const float* u,
                               cudaStream_t s);
cudaError_t launch_moments(const Params& P, const void* pop, float4* M, float* dn, int* status,
                           cudaStream_t s);
cudaError_t launch_ball(const Params& P, const float* dn, float* dG, int* status, cudaStream_t s);
cudaError_t launch_tail(const Params& P, const float* dn, const int* off, const float4* K,
                        int npairs, float4* Ft, cudaStream_t s);
cudaError_t launch_fcs(const Params& P, const void* pin, void* pout, const float4* M,
                       const float* dG, const float4* Ft, cudaStream_t s);
cudaError_t launch_force_out(const Params& P, const float4* M, const float* dG, const float4* Ft,
                             float* F, cudaStream_t s);
cudaError_t launch_moments_out(const Params& P, const float4* M, const float* dG, float* rho,
                               float* u, float* p, cudaStream_t s);
cudaError_t launch_profiles(const Params& P, const float4* M, double* prof, cudaStream_t s);

}  // namespace lbif
