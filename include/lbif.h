/*
 * lbif — lattice Boltzmann for inhomogeneous hard-sphere fluids, one GB300.
 *
 * C ABI of the per-time-step hot path of Melchionna & Marconi, "Lattice
 * Boltzmann method for inhomogeneous fluids" (EPL 2008). Every entry point
 * takes plain pointers and sizes; no C++ or torch type crosses it.
 *
 * Conventions shared by all calls
 *   - Grid: nx * ny * nz nodes, node index idx = (z * ny + y) * nx + x
 *     (x fastest). x and y are periodic; z is periodic or bounded by two
 *     half-way bounce-back walls at z = -1/2 and z = nz - 1/2 (all nz nodes
 *     are fluid). Lattice units: spacing 1, time step 1, m = 1,
 *     k_B T = v_T^2 = c_s^2 = 1/3.
 *   - sigma (hard-sphere diameter) is an even integer number of lattice
 *     spacings (Sec. Methods fixes it so, which puts the axis midpoints on
 *     lattice nodes); odd or non-integer sigma returns LBIF_ERR_UNSUPPORTED.
 *   - Ownership: a handle owns every device buffer it allocates; callers own
 *     all buffers they pass in. Nothing returned aliases caller memory.
 *   - Errors: every call returns 0 (LBIF_OK) or a negative LBIF_ERR_* code
 *     and never aborts; lbif_last_error() gives a message. A divergence
 *     (non-finite or non-positive density, coarse packing fraction >= 1)
 *     is recorded in a device status word and reported as LBIF_ERR_DIVERGED
 *     by the next synchronising call; it is sticky until destroy.
 *   - Streams: work is enqueued on the stream given at creation (NULL = the
 *     legacy default stream). lbif_step is asynchronous; calls that return
 *     host data synchronise that stream.
 *   - Determinism: no atomics on data paths; the same inputs give
 *     bit-identical outputs.
 */
#ifndef LBIF_H
#define LBIF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBIF_OK               0
#define LBIF_ERR_ARG         -1  /* invalid argument */
#define LBIF_ERR_NOMEM       -2  /* device or host allocation failed */
#define LBIF_ERR_CUDA        -3  /* a CUDA runtime call failed */
#define LBIF_ERR_DIVERGED    -4  /* the state became non-physical (sticky) */
#define LBIF_ERR_TIMEOUT     -5  /* a bounded device wait ran out */
#define LBIF_ERR_UNSUPPORTED -6  /* parameters outside what the method defines */
#define LBIF_ERR_IO          -7  /* checkpoint file error */

typedef struct lbif_ctx* lbif_handle; /* opaque, library-owned */

typedef struct { int32_t nx, ny, nz; } lbif_grid;

typedef enum { LBIF_WALL_BOUNCEBACK = 0, LBIF_PERIODIC = 1 } lbif_zbc;
typedef struct { int32_t z; /* lbif_zbc */ } lbif_walls;

/* Forces entering the collisional source (Eq. brey; C1 of Eq. LBHS). */
typedef struct {
    double  body[3];   /* F_e per particle (Eq. uno); force density n F_e   */
    int32_t hs;        /* 1: hard-sphere shell force of Eq. LBHS           */
    int32_t coupling;  /* 1: density-current term of Eq. LBHS              */
    int32_t regularize;/* 1: (1 - exp(-|r - r_w|/sigma)) on that term      */
    int32_t g2_form;   /* 0: g2 as printed in Sec. Methods; 1: Carnahan-Starling */
    int32_t tail;      /* 1: Lennard-Jones mean-field attractive tail       */
    double  eps;       /* tail well depth (k_B T = 1/3 units)               */
    double  rcut;      /* tail cut-off in units of sigma                    */
    int32_t c2;        /* 1: energy source of Eq. C2eq at constant T, added
                          as the isotropic second-order Hermite source
                          w_i C2 (|c_i|^2 - 3 kT) / (6 kT^2) (no mass, no
                          momentum; C2 from the same shell quadrature and
                          interpolants as the force, not regularised)       */
    int32_t shifted;   /* 1: velocity-shifted second-order forcing instead of
                          the first-order source of Sec. Methods: the force
                          F from the moments n, u = j/n as before (explicit),
                          BGK towards f^eq(n, u + F/(2n)), source
                          (1 - 1/(2 tau)) w_i [(c_i - u').F/c_s^2 +
                          (c_i.u')(c_i.F)/c_s^4]. lbif_moments still reports
                          u = j/n (the physical velocity is u + F/(2n), F
                          from lbif_forces). Not with c2. */
} lbif_force;

/* Population storage. Each population is stored as its non-equilibrium part
 * relative to the equilibrium of its own node, h_i = (f_i - f_i^eq(n, u)) /
 * (w_i n), at the moments n, u of the step it belongs to, which the handle
 * keeps in FP32; the equilibrium part, which carries the flow, is never
 * rounded to the storage type. */
#define LBIF_STORE_F32 0 /* h_i in FP32                                         */
#define LBIF_STORE_F16 1 /* 2^8 h_i in FP16 (round to nearest; the factor keeps
                            small parts clear of the FP16 subnormal range)     */

typedef struct {
    int32_t  storage;  /* LBIF_STORE_F32 or LBIF_STORE_F16                     */
    uint64_t seed;     /* initial density noise: n = n0 (1 + noise (2U - 1)),  */
    double   noise;    /*   U from SplitMix64(seed ^ node index)                */
    void*    stream;   /* cudaStream_t to enqueue on; NULL = default stream    */
    int32_t  inplace;  /* 1: the populations live in one buffer (half the
                          memory): direction i of every node moves by c_i
                          slots each step, so each step reads and writes the
                          same slots; 0: two buffers (read one, write the
                          other). Same arithmetic, same results. In place,
                          19 x (nodes of the slits' storage rings, padded)
                          must stay below 2^32 (about 226 M nodes), else
                          LBIF_ERR_UNSUPPORTED.                               */
} lbif_opts;

/* Create a slit (or periodic box) of packing fraction eta = pi sigma^3 n0/6
 * with BGK relaxation time tau (> 1/2) and initialise the populations to the
 * rest equilibrium of the seeded noisy density (Sec. Methods, local
 * equilibrium; Sec. Methods, slit with bounce-back walls). f may be NULL
 * (ideal fluid, no force); o may be NULL (FP32, seed 0, noise 1e-3, default
 * stream). On success *out receives the handle. */
int lbif_create(lbif_handle* out, lbif_grid g, double sigma, double eta, double tau,
                lbif_walls w, const lbif_force* f, const lbif_opts* o);

/* Advance nsteps forward-Euler LB updates (Sec. Methods, update of f_i):
 * moments n, u = j/n; coarse-grained density and g2 field; the shell force
 * of Eq. LBHS (plus body force and tail); BGK collision with source
 * w_i c_i.F/c_s^2; streaming with bounce-back. Asynchronous. */
int lbif_step(lbif_handle h, int64_t nsteps);

/* Same as lbif_step, and also times every kernel class with CUDA events
 * recorded on the handle's stream between launches: kernel_ms[k] receives
 * the total milliseconds of class k over the nsteps (k = 0 moments, 1 ball +
 * g2, 2 tail, 3 force, 4 collide + stream; classes not launched get 0) and
 * launches[k] the number of launches. nk = length of both arrays (>= 5).
 * Class 4 includes the moments of the next step (the pull pass, see
 * lbif_set_fused); class 0 is no longer launched (every state set from
 * outside is an equilibrium whose moments are the given fields). Synchronises
 * at the end. Diagnostics for the benchmark. */
int lbif_step_profiled(lbif_handle h, int64_t nsteps, double* kernel_ms, int64_t* launches,
                       int32_t nk);

/* Density n (nx*ny*nz floats), velocity u (3 planes of nx*ny*nz floats,
 * SoA: u_x then u_y then u_z) and local pressure p = k_B T n + the static
 * collisional part (k_B T sigma^3/6) 4 pi sum_q W_q g2_q n n_q (bulk limit:
 * Sec. Theory, p_bulk) of the current populations. Any pointer may be NULL.
 * on_device = 1: pointers are device memory; 0: host memory. Synchronises. */
int lbif_moments(lbif_handle h, float* rho, float* u, float* pressure, int32_t on_device);

/* Total force density F / n0 (3 SoA planes) of the current state, as used by
 * the next step (body + hard sphere + tail). Diagnostics; synchronises. */
int lbif_forces(lbif_handle h, float* F, int32_t on_device);

/* Re-initialise the populations to f_eq(n, u) of given fields (same layout
 * as lbif_moments; u may be NULL = 0) and reset the step counter. The stored
 * non-equilibrium parts become 0 and the given fields are the moments of
 * step 0 (no moments pass); u NULL and an explicit u = 0 give the same state,
 * bit for bit. on_device = 0: host pointers, copied in on the handle's
 * stream through the handle's second population buffer (rho) and its
 * scratch (u). Synchronises. */
int lbif_set_fields(lbif_handle h, const float* rho, const float* u, int32_t on_device);

/* FP64 x,y-averaged profiles n(z), u_x(z) (nz doubles each; either may be
 * NULL), total mass and momentum (out4 = {M, Jx, Jy, Jz}; may be NULL), from
 * a deterministic reduction on the device (per thread exact FP32 two-sum
 * pairs, about 48 bits; FP64 across threads in a fixed order). Synchronises. */
int lbif_profiles(lbif_handle h, double* n_z, double* ux_z, double* out4);

/* Steady-state residual over the steps since the previous call:
 *   R = max over {n(z), u_x(z)} of ||p(t) - p(t0)||_2 / ((t - t0) ||p(t)||_2),
 * FP64; R = +inf on the first call. mass/mom may be NULL. Synchronises. */
int lbif_residual(lbif_handle h, double* r, double* mass, double mom[3]);

/* Steps taken since creation (or the last lbif_set_fields). */
int lbif_time(lbif_handle h, int64_t* t);

/* Device status word (0 = healthy; bit 0 divergence). Synchronises. */
int lbif_status(lbif_handle h, int32_t* status);

/* Checkpoint: write / read the stored populations and the moment fields
 * they refer to (dn = n/n0 - 1, u; storage tag, grid, step count) to / from a
 * host file; a resumed run continues bit for bit. lbif_load requires a handle
 * of the same grid, sigma and storage. */
int lbif_save(lbif_handle h, const char* path);
int lbif_load(lbif_handle h, const char* path);

/* ---- ensemble of slits ---------------------------------------------------
 * Many independent slits of one sigma and lateral size nx x ny, each with its
 * own width H[s] (nodes along z), packing fraction eta[s], body force F[s]
 * (per particle, along x) and relaxation time tau[s], advanced together: they
 * are stacked along z with hw >= sigma planes of "outside" (n = 0) between
 * them, so every stencil of the step (ball, shell, streaming, bounce-back)
 * sees only its own slit, and one launch per kernel covers all of them.
 * f gives the force model (its body[] is ignored); o as for lbif_create, but
 * with o->stream NULL the handle creates and owns a non-blocking stream
 * (needed for graph capture). lbif_step / lbif_moments / lbif_profiles /
 * lbif_save / lbif_load work on the stacked grid (gap planes read as 0).
 * With o->inplace = 1 each slit's populations occupy only its own ring of
 * H + 1 planes (the gap planes hold fields but no populations), which is
 * both half the memory and the faster layout for ensembles. */
int lbif_batch_create(lbif_handle* out, int32_t nslits, const int32_t* H, const double* eta,
                      const double* F, const double* tau, double sigma, int32_t nx, int32_t ny,
                      const lbif_force* f, const lbif_opts* o);

/* Number of slits, first plane of each slit in the stacked grid (zlo[nslits],
 * may be NULL) and the number of fluid nodes. */
int lbif_batch_info(lbif_handle h, int32_t* nslits, int32_t* zlo, int64_t* nodes);

/* Re-initialise every slit to the local equilibrium of x,y-uniform profiles:
 * n_z[s*hmax + j], ux_z[s*hmax + j] (host arrays; ux_z may be NULL = 0) for
 * the j-th plane of slit s, j < H[s] (entries j >= H[s] are ignored). Resets
 * the step counter. Used to seed slits from a predicted steady state. */
int lbif_batch_seed(lbif_handle h, const float* n_z, const float* ux_z, int32_t hmax);

/* Advance all slits, check_every steps per CUDA-graph replay (rounded up to
 * even), until every slit's residual (lbif_residual's definition over its own
 * x,y-averaged profiles, with t - t0 = check_every) is below tol, or
 * max_steps. Converged slits are frozen (their kernels exit at once) while the
 * others continue. With patience > 0 a slit whose residual has not improved
 * for patience consecutive checks is frozen too: its rounding floor (FP32 /
 * FP16 state) lies above tol. steps_taken[s] (may be NULL) = steps at which
 * slit s met tol, -1 if it did not within max_steps, -2 if it diverged, -3 if
 * it stalled; residual[s] (may be NULL) = the smallest residual it reached. */
int lbif_batch_run(lbif_handle h, double tol, int64_t max_steps, int32_t check_every,
                   int32_t patience, int64_t* steps_taken, double* residual);

/* FP64 x,y-averaged profiles of every slit, n_z / ux_z[s*hmax + j] (host
 * arrays, either may be NULL; zero beyond H[s]). Synchronises. */
int lbif_batch_profiles(lbif_handle h, double* n_z, double* ux_z, int32_t hmax);

/* How a step applies collision and streaming (Sec. Methods: BGK collision
 * with the first-order source, streaming, half-way bounce-back). Every step
 * runs one pass: each node gathers the populations streaming into it (pull
 * form), applies the collision of their source node, and forms the moments
 * n, u of the next step from the values it holds, so the populations are
 * read and written once per step (32 x 4 node tiles marching in z; grids
 * with nx < 32 or ny < 4 run the same arithmetic one node per thread, with
 * identical results). Populations are stored as their non-equilibrium parts
 * relative to the equilibrium of their own node, which this pull form
 * decodes from the staged moments of the source node; the earlier two-pass
 * step (push streaming, then a moments pass) could not, and is retired.
 * lbif_set_fused(h, 1) is accepted and changes nothing; lbif_set_fused(h, 0)
 * returns LBIF_ERR_UNSUPPORTED. LBIF_ERR_ARG for a NULL handle or fused not
 * 0 or 1. */
int lbif_set_fused(lbif_handle h, int32_t fused);
/* The pass in use: always *fused = 1. */
int lbif_get_fused(lbif_handle h, int32_t* fused);

/* Self-test of the failure path of the bounded device waits (the paper has no
 * counterpart). The kernels that wait on an mbarrier for a tile copy give up
 * after a fixed number of polls, record a status bit, and return, so that a
 * lost copy surfaces as LBIF_ERR_TIMEOUT instead of a hang. This call runs the
 * same wait on a barrier that nothing completes, with `polls` polls (>= 1),
 * on the current device's default stream, and synchronises. *timed_out = 1
 * and LBIF_ERR_TIMEOUT when the wait ran out (always, unless the device is
 * broken); LBIF_ERR_ARG for polls < 1 or a NULL pointer. The CUDA context
 * stays usable afterwards. */
int lbif_selftest_wait(int64_t polls, int32_t* timed_out);

/* Time the candidate launch shapes of the step's kernels on this handle's
 * current state (trials launches each) and keep the fastest: the ball
 * kernel's CTA target and its plane staging (1 = tensor-memory-accelerator
 * copies, 0 = plain loads), the force kernel's tile-group edge, and the pull
 * pass's z planes per CTA segment (8, 16, 32) and its gathers (plain; the
 * next plane's populations loaded while the current one is collided; or the
 * per-direction source boxes of each tile copied into shared memory one plane
 * ahead by the tensor-memory accelerator, two-buffer handles whose x rows
 * are a multiple of 16 bytes). Trials
 * write only buffers the step overwrites, so the state is unchanged, and no
 * choice changes the arithmetic (results are bit-identical). Chosen values
 * (each may be NULL): ball CTA target, force tile-group edge in nodes, ball
 * staging; lbif_get_shapes gives all of them. */
int lbif_autotune(lbif_handle h, int32_t trials, int32_t* ball_want, int32_t* force_group,
                  int32_t* ball_staging);
/* The launch shapes in use: shapes[0] ball CTA target (0 = default),
 * [1] force tile-group edge (0 = default), [2] ball staging (1 = tensor-
 * memory accelerator), [3] pull-pass z planes per segment (0 = default 16),
 * [4] pull-pass gathers (0 plain, 1 prefetched, 2 tensor-memory accelerator). */
int lbif_get_shapes(lbif_handle h, int32_t shapes[5]);
/* Set the launch shapes (same order and meaning as lbif_get_shapes) instead of
 * timing them; no shape changes the arithmetic. Accepted: [0] 0 or 1..2^20,
 * [1] 0 or 1..2^20, [2] 0/1, [3] 0 or 1..2^20, [4] 0/1/2. LBIF_ERR_ARG for a value
 * out of range; LBIF_ERR_UNSUPPORTED for [2] = 1 or [4] = 2 on a handle
 * without the tensor maps they read (none is changed then). */
int lbif_set_shapes(lbif_handle h, const int32_t shapes[5]);

/* ---- warm-start network -------------------------------------------------
 * A multilayer perceptron nin -> nhidden layers of width `hidden` (GELU, erf
 * form) -> nout, mapping slit parameters to predicted steady profiles; it only
 * seeds populations (lbif_batch_seed), the lattice Boltzmann iteration always
 * runs to convergence. Products run on the tensor cores with bfloat16
 * operands and FP32 accumulation; master weights, Adam moments and all
 * element-wise work are FP32. Parameters are one flat FP32 vector: for each
 * layer W (out x in, row-major) then b (out). Widths <= 256. The paper has no
 * counterpart: the network is an added way to choose the starting state.
 * Errors: LBIF_ERR_ARG for bad widths, sizes or NULL pointers (checked before
 * any device work), LBIF_ERR_NOMEM, LBIF_ERR_CUDA, LBIF_ERR_UNSUPPORTED for a
 * product outside the kernel's shapes, LBIF_ERR_TIMEOUT when a bounded wait of
 * the tensor-core kernel ran out. The handle owns its device memory; arrays
 * passed in stay the caller's. All calls run on the handle's stream. */
typedef struct lbif_mlp_ctx* lbif_mlp;

int lbif_mlp_create(lbif_mlp* out, int32_t nin, int32_t hidden, int32_t nhidden, int32_t nout,
                    int32_t max_batch, void* stream);
int64_t lbif_mlp_num_params(lbif_mlp m);
/* host arrays of lbif_mlp_num_params floats; set_params also resets Adam */
int lbif_mlp_set_params(lbif_mlp m, const float* params);
int lbif_mlp_get_params(lbif_mlp m, float* params);
/* Y (batch x nout) = network(X (batch x nin)); on_device selects device or
 * host pointers. Synchronises. */
int lbif_mlp_forward(lbif_mlp m, const float* X, int32_t batch, float* Y, int32_t on_device);
/* Loss = sum(mask (Y - T)^2) / sum(mask) and its gradient (flat, like the
 * parameters; grads may be NULL). */
int lbif_mlp_gradients(lbif_mlp m, const float* X, const float* T, const float* mask, int32_t batch,
                       float* grads, double* loss, int32_t on_device);
/* One Adam step (bias-corrected) on that loss; *loss receives it. */
int lbif_mlp_train_step(lbif_mlp m, const float* X, const float* T, const float* mask, int32_t batch,
                        float lr, float beta1, float beta2, float eps, double* loss, int32_t on_device);
int lbif_mlp_destroy(lbif_mlp m);
const char* lbif_mlp_last_error(lbif_mlp m);

/* ---- profiles without allocation ------------------------------------------
 * No counterpart in the paper: an operational entry point. It gives the same
 * FP64 x,y-averaged profiles n(z), u_x(z) and totals {mass, momentum} as
 * lbif_profiles, but of fields the caller holds - rho (nx*ny*nz floats) and
 * u (3 SoA planes), device pointers, layout as lbif_moments - and it
 * allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
 * It is meant for callers that cannot allocate device memory when they need
 * the profiles: services whose device memory is reserved up front by their
 * own allocator (a further cudaMalloc would fail or fragment it), and loops
 * that must keep a fixed memory footprint.
 * Its scratch is a fixed 320 KB array in the library's device image, which
 * every GPU that loads the library keeps until the process exits; nz above
 * 8192 is rejected with LBIF_ERR_UNSUPPORTED. All calls share that array:
 * calls that overlap on the GPU (other streams, other threads) race on it.
 * Every call overwrites what it uses, nothing needs clearing. The first call
 * on a device looks the array's device address up (cudaGetSymbolAddress, with
 * that device current), and so does the first call after the device's context
 * changed (a reset reloads the image elsewhere); make that first call before
 * any stream capture.
 * n_z, ux_z (nz doubles) and out4 are host pointers (any may be NULL); work is
 * enqueued on `stream` (cudaStream_t, NULL = default) and synchronised. On
 * error, lbif_noalloc_last_error() gives a message. */
int lbif_field_profiles_noalloc(const float* rho, const float* u, int32_t nx, int32_t ny,
                                int32_t nz, double* n_z, double* ux_z, double* out4,
                                void* stream);
const char* lbif_noalloc_last_error(void);

int lbif_destroy(lbif_handle h);

/* Message of the last error of a handle; NULL handle = last global error
 * (e.g. of a failed lbif_create). Never NULL. */
const char* lbif_last_error(lbif_handle h);

#ifdef __cplusplus
}
#endif
#endif /* LBIF_H */
