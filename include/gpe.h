/*
 * gpe.h -- C ABI of libgpeshell: the finite-difference Gross-Pitaevskii (GPE)
 * step on a selectively sampled ("semi-structured") Cartesian grid, on one
 * NVIDIA GB300 GPU (sm_103a).
 *
 * Method: Beregi, Gerent, Lundblad, "Efficient simulation of Bose-Einstein
 * condensates in nontrivial topologies".  Units hbar = m = 1.  The problem is
 * the paper's own statement of it (Sec. II): a potential V on a Cartesian grid
 * and a cutoff select a region of interest; psi is stepped in imaginary time
 * (Eqs. (6)-(7), ground state with renormalisation to N, Eq. (3)) or in real
 * time (Eq. (8), explicit Runge-Kutta); norm, energy and chemical potential are
 * reported.
 *
 * Conventions (every call):
 *  - Every function returns GPE_OK (0) or a negative GPE_ERR_* code; on error
 *    gpe_last_error() returns a one-line description (thread-local).  No C++
 *    exception crosses this ABI.
 *  - Handles (gpe_grid, gpe_state, gpe_batch, gpe_tape) are opaque, created and
 *    freed by the library, and bound to the CUDA device that was current when
 *    they were created.  Calls on a handle must be made with that device
 *    current.
 *  - Host pointers are read or written before the call returns and are never
 *    retained.  Device pointers are borrowed for the duration of the call (the
 *    copy is ordered on `stream`; the caller keeps the memory alive until the
 *    stream has passed it).
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Calls documented as asynchronous only enqueue work on it; calls
 *    that return results on the host synchronise that stream.
 *  - Complex arrays are interleaved (re, im) pairs: complex64 = two float32,
 *    complex128 = two float64.
 *  - Dense box arrays are laid out x fastest: cell (i, j, k) at linear index
 *    i + nx*(j + ny*k); cell centres at (x0 + i*hx, y0 + j*hy, z0 + k*hz).
 *  - The compact layout is the library's device layout: bricks of bx*by*bz
 *    lattice cells in brick-list order; a brick is cut into segments of 4
 *    cells along x (local cell l = x + bx*(y + by*z), segment l/4) and stores,
 *    in segment order, exactly the segments that hold an active cell, 4
 *    entries each.  Cells of stored segments that are not active hold zero.
 *    Length n_packed = 4 * (number of stored segments).
 */
#ifndef GPE_H
#define GPE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
enum {
    GPE_OK = 0,
    GPE_ERR_ARG = -1,           /* invalid argument (checked before any GPU work) */
    GPE_ERR_CUDA = -2,          /* a CUDA runtime call failed */
    GPE_ERR_OOM = -3,           /* device allocation failed */
    GPE_ERR_NONFINITE = -4,     /* a reduction saw NaN or Inf in psi */
    GPE_ERR_UNSTABLE = -5,      /* dt beyond the integrator's stability bound */
    GPE_ERR_NOT_CONVERGED = -6, /* ground-state iteration hit max_steps */
    GPE_ERR_STATE = -7          /* handle in the wrong state for this call */
};

typedef void *gpe_stream; /* cudaStream_t */

typedef struct gpe_grid gpe_grid;
typedef struct gpe_state gpe_state;
typedef struct gpe_batch gpe_batch;
typedef struct gpe_tape gpe_tape;

/* Library version (major*10000 + minor*100 + patch). */
int gpe_version(void);

/* Copy the calling thread's last error message into buf (NUL-terminated,
 * truncated to n bytes).  Returns the length of the full message. */
int gpe_last_error(char *buf, size_t n);

/* Number of CUDA kernels this library has launched in this process
 * (diagnostics; counts enqueued launches, including those captured into
 * CUDA graphs at capture time only). */
int gpe_launch_count(uint64_t *out);

/* Arithmetic roof of this GPU (diagnostics; the paper has no counterpart): the
 * fused multiply-add throughput of the CUDA cores in FP64 (dtype GPE_F64) or
 * FP32 (GPE_F32), measured by one launch of independent FMA chains on every
 * SM (iters x 16 x 8 FMAs per thread, about 1 s for FP64 at iters = 20000)
 * timed with CUDA events.  *tflops = 2 flops per FMA / elapsed time,
 * *seconds = that time.  The complex128 step is bound by this FP64 rate, not
 * by HBM.  GPE_ERR_ARG for iters outside [1, 2^24].  Synchronous. */
int gpe_fma_peak(int dtype, int iters, double *tflops, double *seconds);

/* ------------------------------------------------------------------ grids */
/* Cartesian bounding box.  (x0, y0, z0) is the centre of cell (0, 0, 0). */
typedef struct gpe_box {
    int64_t nx, ny, nz;
    double hx, hy, hz;
    double x0, y0, z0;
} gpe_box;

enum { GPE_MASK_CELL = 0,   /* active = cells with V < V_cut (Sec. II A) */
       GPE_MASK_BRICK = 1 }; /* active = every in-box cell of a brick holding
                                at least one cell with V < V_cut (Sec. II B) */
enum { GPE_ORDER_ZMAJOR = 0, GPE_ORDER_MORTON = 1 };

/* Step schedules: STAGED (default) launches one kernel per stage, the
 * paper's scheme (Sec. II B); WAVE runs every stage of a time step in one
 * persistent launch, ordering (stage, chunk) tasks so that a stage of a chunk
 * starts once the previous stage has finished on every chunk its stencil
 * touches, which keeps the intermediate stage states in L2 on grids whose
 * skewed window fits there; WAVE2 runs an RK4 step as two such launches of
 * two stages each (stages 0-1, then 2-3), a window of a third of WAVE's
 * (imaginary-time steps have two stages: WAVE2 is WAVE there).  PAIR runs
 * the RK4 step of gpe_step_real as two launches, stages 0+1 and stages 2+3,
 * each brick recomputing the first stage of a pair on its one-cell face halo
 * so that the middle stage never leaves shared memory (64 instead of 112
 * bytes of compulsory traffic per stored cell in complex64); it runs the
 * imaginary-time step of a complex state as one launch, each brick
 * recomputing the first Euler substep on its one-cell face halo (20 instead
 * of 40 bytes per stored cell); the other calls run STAGED on such a grid.
 * All four give bit-identical real-time results; PAIR's imaginary-time step
 * sums the norm in another order, so its renormalisation factor can differ
 * from STAGED's in the last bit. */
enum { GPE_SCHED_STAGED = 0, GPE_SCHED_WAVE = 1, GPE_SCHED_WAVE2 = 2, GPE_SCHED_PAIR = 3 };

/* Grid options.  Brick shape (bx, by, bz) must be one of 8x8x8 (default when
 * all three are 0), 8x8x4, 8x4x4.  chunk = bricks per wavefront task
 * (0: about 2048 lattice cells).  stencil = 7 (default, also 0): the 7-point
 * Laplacian (Eq. (B1)); 19: the 19-point higher-order compact Laplacian of
 * App. B, which also reads the 12 edge neighbours of a cell.  A 19-point grid
 * runs the staged schedule for gpe_step_real (RK4), gpe_step_imag,
 * gpe_observables and gpe_ground_state; the other step calls refuse it
 * (GPE_ERR_ARG). */
typedef struct gpe_grid_opts {
    int32_t bx, by, bz;
    int32_t mask_mode; /* GPE_MASK_* */
    int32_t order;     /* GPE_ORDER_* : order of the brick list in memory */
    int32_t sched;     /* GPE_SCHED_* */
    int32_t chunk;
    int32_t stencil;   /* 0 or 7, or 19 */
} gpe_grid_opts;

enum { GPE_F64 = 1, GPE_F32 = 2 };   /* element type of a real input array */

/* Analytic potentials evaluated on the device (needed for boxes whose dense
 * potential does not fit in memory):
 *   GPE_POT_HARMONIC        V = 1/2 (p0^2 x^2 + p1^2 y^2 + p2^2 z^2)
 *   GPE_POT_ELLIPSOID_SHELL V = 1/2 p0^2 (rho - 1)^2,
 *                           rho = sqrt(x^2/p1^2 + y^2/p2^2 + z^2/p3^2)
 * Unused parameters must be zero. */
enum { GPE_POT_HARMONIC = 1, GPE_POT_ELLIPSOID_SHELL = 2 };
typedef struct gpe_potential {
    int32_t kind;
    int32_t reserved;
    double p[8];
} gpe_potential;

/* Build a grid from a dense potential V (nx*ny*nz values of type V_dtype, on
 * the host or the device) and a cutoff: the region of interest is the set of
 * cells with V < V_cut (Sec. II A, region of interest from the Thomas-Fermi
 * estimate of Eq. (5); the caller picks V_cut, e.g. 5 mu).  The active cells
 * are compacted into bricks (Sec. II B), ordered by opts->order, with a
 * brick-neighbour table; absent neighbours read as psi = 0 (rows and columns
 * deleted from the Laplacian, Sec. II A).  Potential slot 0 holds V.
 * opts may be NULL (8x8x8, cell mask, Morton order).  Synchronous. */
int gpe_grid_create_dense(const gpe_box *box, const void *V, int V_dtype,
                          int V_on_device, double V_cut,
                          const gpe_grid_opts *opts, gpe_grid **out,
                          gpe_stream stream);

/* Same, with V evaluated on the device from an analytic description. */
int gpe_grid_create_analytic(const gpe_box *box, const gpe_potential *pot,
                             double V_cut, const gpe_grid_opts *opts,
                             gpe_grid **out, gpe_stream stream);

/* Default brick order is z-major (bricks sorted by z, then y, then x); it
 * bounds how far apart neighbouring bricks are in memory, which the wavefront
 * schedule needs.  Morton order is offered for the staged schedule. */

/* Grid for a potential ramp V(t) = (1 - s) V0 + s V1 (Sec. V: linear
 * interpolation between precomputed potentials).  With the cutoff blended the
 * same way, the union over s in [0, 1] of {V(s) < cut(s)} is exactly
 * {V0 < cut0} U {V1 < cut1}; that union is the region of interest.  Slot 0
 * holds V0 and slot 1 holds V1.  Synchronous. */
int gpe_grid_create_blend(const gpe_box *box, const gpe_potential *pot0,
                          double cut0, const gpe_potential *pot1, double cut1,
                          const gpe_grid_opts *opts, gpe_grid **out,
                          gpe_stream stream);

/* The same union region for two dense potentials V0, V1 (nx*ny*nz values
 * each, both of type V_dtype and both on the host or both on the device, as
 * in gpe_grid_create_dense): active cells are those with V0 < cut0 or
 * V1 < cut1; slot 0 holds V0 and slot 1 holds V1.  Synchronous. */
int gpe_grid_create_blend_dense(const gpe_box *box, const void *V0,
                                const void *V1, int V_dtype, int V_on_device,
                                double cut0, double cut1,
                                const gpe_grid_opts *opts, gpe_grid **out,
                                gpe_stream stream);

/* Replace potential slot 0 or 1 with a dense potential (same layout as
 * gpe_grid_create_dense); the region of interest is unchanged.  Synchronous. */
int gpe_grid_set_potential(gpe_grid *grid, int slot, const void *V,
                           int V_dtype, int V_on_device, gpe_stream stream);

typedef struct gpe_grid_info {
    int64_t n_active;  /* cells in the region of interest */
    int64_t n_bricks;
    int64_t n_stored;  /* lattice cells of the bricks: n_bricks * bx*by*bz */
    int64_t n_packed;  /* length of the compact layout (active cells + padding) */
    int32_t bx, by, bz, mask_mode;
    int32_t order, n_slots; /* number of potential slots filled (1 or 2) */
    double v_max;      /* max of |V| over active cells, all slots */
    gpe_box box;
} gpe_grid_info;

int gpe_grid_get_info(const gpe_grid *grid, gpe_grid_info *out);

/* Host copies of the layout: brick origins in cells (3 int32 per brick,
 * i0 j0 k0), the neighbour table (6 int32 per brick: -x +x -y +y -z +z, -1 =
 * absent; may be NULL), the active-cell bit mask (n_stored/32 words, bit l of
 * word w = lattice cell 32w + l of the brick list), and potential slot `slot`
 * in the compact layout (n_packed doubles; slot 0 holds +inf at the inactive
 * cells of stored segments, which is how the kernels tell them apart).
 * Synchronous. */
int gpe_grid_bricks(const gpe_grid *grid, int32_t *origins, int32_t *nbr);
int gpe_grid_mask(const gpe_grid *grid, uint32_t *bits);
int gpe_grid_potential(const gpe_grid *grid, int slot, double *V);

int gpe_grid_destroy(gpe_grid *grid);

/* Thomas-Fermi chemical potential (Sec. II A, Eq. (5)): the mu at which
 * sum over the box of max((mu - V)/g, 0) dV equals N.  That sum is convex and
 * piecewise linear in mu; Newton's method from above (one pass over the box
 * per iterate, typically under ten) ends on the exact root of the final
 * linear piece.  GPE_ERR_ARG for g <= 0, N <= 0 or a non-finite V.
 * Synchronous. */
int gpe_tf_mu_dense(const gpe_box *box, const void *V, int V_dtype,
                    int V_on_device, double g, double N, double *mu,
                    gpe_stream stream);
int gpe_tf_mu_analytic(const gpe_box *box, const gpe_potential *pot,
                       double g, double N, double *mu, gpe_stream stream);

/* ------------------------------------------------------------------ states */
enum { GPE_C128 = 1, GPE_C64 = 2, GPE_R64 = 3, GPE_R32 = 4 };
enum { GPE_LAYOUT_DENSE = 0, GPE_LAYOUT_COMPACT = 1 };

/* A wavefunction on a grid, complex128 or complex64 (bulk precision).  The
 * real types GPE_R64 / GPE_R32 hold a real-valued wavefunction for
 * imaginary-time work: the imaginary-time step keeps a real wavefunction
 * real, so half the bytes suffice (Sec. II A).  Real states support load,
 * store, copy, remap, gpe_step_imag, gpe_observables, gpe_ground_state and
 * batches; the calls that need complex values (real-time steps, overlaps,
 * ramp gradients) refuse them with GPE_ERR_ARG.  Load and store use arrays
 * of double / float.  The state keeps a reference to the grid: destroy
 * states before their grid. */
int gpe_state_create(gpe_grid *grid, int dtype, gpe_state **out);

/* Load psi from a dense box array (inactive cells are ignored) or from the
 * compact layout (inactive slots are forced to zero).  Asynchronous for device
 * input; host input is staged through the library and the call returns once
 * the host buffer has been read. */
int gpe_state_load(gpe_state *st, const void *psi, int layout, int on_device,
                   gpe_stream stream);

/* Store psi to a dense box array (cells outside the region are zero) or to the
 * compact layout.  Asynchronous for device output; synchronous for host. */
int gpe_state_store(const gpe_state *st, void *psi, int layout, int on_device,
                    gpe_stream stream);

/* dst <- src (same grid and dtype).  Asynchronous. */
int gpe_state_copy(gpe_state *dst, const gpe_state *src, gpe_stream stream);

/* Remap a state onto another grid over the same box: the regrid between ramp
 * stages of Sec. V (the region of interest is selected again and the
 * wavefunction remapped between the old and new grids).  Every cell active
 * in both grids takes src's value; cells active only in dst's grid become 0;
 * src's cells outside dst's region are dropped (renormalise afterwards if
 * the norm should be kept).  The grids must share box sizes, spacings and
 * origin (bit-identical gpe_box); brick shapes and orders may differ.  Same
 * dtype, distinct states, same device.  GPE_ERR_ARG otherwise.
 * Asynchronous. */
int gpe_state_remap(gpe_state *dst, const gpe_state *src, gpe_stream stream);

/* Failure detection self-test: one warp waits (with the same bounded wait the
 * wavefront schedule uses) for a completion stamp that nothing sets; the wait
 * gives up after limit_s seconds (0 < limit_s <= 10) and reports it.  Sets
 * *timed_out (1 expected) and *waited_s (may be NULL).  No GPU fault or hang
 * is involved: the kernel returns and the context stays usable.  Synchronous. */
int gpe_wait_selftest(double limit_s, int *timed_out, double *waited_s);

/* Step loops on the staged schedule are captured in CUDA graphs of
 * steps_per_graph steps (default 32; 0 disables) and replayed, when the
 * stream is not the legacy default stream and a call asks for at least that
 * many steps; each distinct parameter set is captured once per state.  The
 * wavefront schedule always launches directly. */
int gpe_state_set_graph(gpe_state *st, int steps_per_graph);

/* Device pointer of the compact psi array (borrowed; valid until destroy). */
int gpe_state_device_ptr(gpe_state *st, void **dptr);

int gpe_state_destroy(gpe_state *st);

/* ------------------------------------------------------------------ steps */
/* Imaginary time (Sec. II A, Eqs. (6)-(7)).  Each step, in the paper's order:
 *  psi <- psi exp(-V dt/2) (1 - g|psi|^2 dt/2)    (diagonal half step)
 *  psi <- psi - (dt/2) T psi, twice               (kinetic: two Euler steps)
 *  psi <- psi exp(-V dt/2) (1 - g|psi|^2 dt/2)    (diagonal half step)
 *  psi <- psi sqrt(N / sum |psi|^2 dV)            (renormalise, Eq. (3))
 * with T = -1/2 Laplacian (7 point, Eq. (B1)) and V from slot 0.  The
 * renormalisation factor is computed on the device in FP64 and applied when
 * the next step loads psi (Sec. II B); the state is fully normalised when the
 * call's work completes.  Asynchronous.  GPE_ERR_UNSTABLE if
 * dt * sum_e 2/h_e^2 > 4 (the Euler substep would amplify the top mode). */
typedef struct gpe_imag_params {
    double g, dt, N;
} gpe_imag_params;

int gpe_step_imag(gpe_state *st, const gpe_imag_params *p, int64_t nsteps,
                  gpe_stream stream);

/* Real time (Sec. II A, Eq. (8)) with the classic RK4 method in the
 * memory-optimised stage form of App. A:
 *   y2 = y0 + dt/2 f(t, y0);  y3 = y0 + dt/2 f(t + dt/2, y2);
 *   y4 = y0 + dt f(t + dt/2, y3);
 *   y1 = -y0/3 + y2/3 + 2 y3/3 + y4/3 + dt/6 f(t + dt, y4)
 * f(t, y) = -i (T + V(t) + g|y|^2) y.  V(t) = V0 (GPE_V_STATIC) or
 * (1 - s(t)) V0 + s(t) V1 (GPE_V_BLEND) with s piecewise linear through
 * n_knots (2..16) values at uniform times on [0, T_ramp], constant outside.
 * t0 is the time at the start of the first step.  Asynchronous.
 * GPE_ERR_UNSTABLE if dt (sum_e 2/h_e^2 + v_max) exceeds the integrator's
 * imaginary-axis limit for the linear part (below). */
/* Integrators: the classic RK4 (default), Heun's third-order method RKHE3 and
 * the fifth-order solution of the Cash-Karp pair RKCK, the three schemes whose
 * memory-optimised stage forms App. A tabulates (Eqs. (A6)-(A7)):
 *   y^(i+1) = sum_j a*_ij y^(j) + dt a_{i+1,i} f(t + c_i dt, y^(i)),
 *   y1 = sum_j b*_j y^(j) + dt b_s f(t + c_s dt, y^(s)).
 * Imaginary-axis limits of dt lambda_max: RK4 2 sqrt(2), RKHE3 sqrt(3).  The
 * RKCK stability function exceeds 1 on the whole imaginary axis (~1 + 1.39e-4
 * y^6); its steps are accepted up to y = 0.43, a growth of at most 1e-6 per
 * step. */
enum { GPE_RK4 = 0, GPE_RKHE3 = 1, GPE_RKCK = 2 };
enum { GPE_V_STATIC = 0, GPE_V_BLEND = 1 };
#define GPE_MAX_KNOTS 16
typedef struct gpe_real_params {
    double g, dt;
    int32_t integrator; /* GPE_RK4, GPE_RKHE3, GPE_RKCK */
    int32_t potential;  /* GPE_V_* */
    int32_t n_knots, reserved;
    double T_ramp;
    double knots[GPE_MAX_KNOTS];
} gpe_real_params;

int gpe_step_real(gpe_state *st, const gpe_real_params *p, int64_t nsteps,
                  double t0, gpe_stream stream);

/* ------------------------------------------------------------------ observables */
/* FP64 reductions over the active cells (products in the state's precision,
 * each 4-cell segment's terms summed in that precision, the segment sums
 * accumulated in FP64 in a fixed order):
 *   norm   = sum |psi|^2 dV                           (Eq. (3))
 *   e_kin  = sum Re(conj(psi) T psi) dV
 *   e_pot  = sum V |psi|^2 dV,  V = (1 - s_blend) V0 + s_blend V1
 *   e_int  = sum (g/2) |psi|^4 dV
 *   energy = e_kin + e_pot + e_int
 *   mu     = (e_kin + e_pot + 2 e_int) / norm   (Eq. (1) projected on psi)
 *   nonfinite = number of active cells holding NaN or Inf.
 * Synchronous; returns GPE_ERR_NONFINITE (with *out filled) when
 * nonfinite > 0. */
typedef struct gpe_obs {
    double norm, energy, mu, nonfinite, e_kin, e_pot, e_int;
} gpe_obs;

int gpe_observables(const gpe_state *st, double g, double s_blend,
                    gpe_obs *out, gpe_stream stream);

/* Real-time steps with an observables trace: nsteps steps as gpe_step_real
 * (same parameters, from time t0), with the observables of gpe_observables
 * taken after every `every` steps and after the last one (potential energy
 * at s(t) of that time for a ramp).  log (host, ceil(nsteps / every)
 * entries) receives them in order and *n_logged how many were written.
 * A trace point that finds a non-finite cell ends the run there with
 * GPE_ERR_NONFINITE (that entry included).  The same steps and the same
 * reductions as separate calls, so the results are bit-identical to them.
 * Synchronous at each trace point. */
int gpe_step_real_traced(gpe_state *st, const gpe_real_params *p,
                         int64_t nsteps, double t0, int64_t every,
                         gpe_obs *log, int64_t *n_logged, gpe_stream stream);

/* out = <a|b> = sum conj(a) b dV as (re, im).  Synchronous. */
int gpe_overlap(const gpe_state *a, const gpe_state *b, double out[2],
                gpe_stream stream);

/* Overlap <a|b> = sum conj(a) b dV of two caller-owned device arrays of n
 * complex values (dtype GPE_C128 or GPE_C64), for callers that cannot
 * allocate device memory when they need the result: for example a host
 * application whose memory pool already holds the device's free memory, or a
 * loop that must not call cudaMalloc/cudaFree (they can synchronise the device
 * and stall other streams).  The paper has no counterpart; it is a service of
 * this library.  Entries of a and b outside the region of interest must be
 * zero (as in a state's compact array, see gpe_state_device_ptr).
 * Allocates nothing: the per-block FP64 partial sums live in a fixed array of
 * 512 KiB compiled into the library, which every GPU that loads the library
 * keeps until the process exits.  Limit: n <= 268,435,456 (one reduction block
 * per 8192 elements, at most 32768 blocks); larger n returns GPE_ERR_ARG.  The
 * first call on each device looks up that array's device address (and looks it
 * up again after the device's CUDA context has been destroyed and made anew,
 * e.g. by cudaDeviceReset), so make the first call before capturing any
 * stream.  All calls share the array: calls whose work overlaps on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  Writes out[0..1] (re, im) on the host; synchronous: the call waits
 * on `stream` for its result before it returns. */
int gpe_overlap_noalloc(const void *a, const void *b, int64_t n, int dtype,
                        double dV, double out[2], gpe_stream stream);

/* Imaginary-time ground state (Sec. III: iterate to a tolerance): gpe_step_imag
 * in blocks of check_every steps until |mu_n - mu_{n-1}| < tol_dmu between two
 * checks.  *steps_done and *obs (may be NULL) report the last check.
 * GPE_ERR_NOT_CONVERGED after max_steps.  Synchronous. */
int gpe_ground_state(gpe_state *st, const gpe_imag_params *p, double tol_dmu,
                     int64_t check_every, int64_t max_steps,
                     int64_t *steps_done, gpe_obs *obs, gpe_stream stream);

/* ------------------------------------------------------------------ batches */
/* Many independent shells in one persistent launch (one launch of each kernel
 * covers every shell of the batch).  The states (complex or real) must share
 * the state type and brick shape; their grids may differ in size, spacing
 * and potential.  The batch copies the states' tables and keeps them alive;
 * destroy the batch before the states' grids. */
int gpe_batch_create(gpe_state *const *states, int n, gpe_batch **out);

/* Imaginary-time ground states of every shell of the batch (Sec. II A,
 * Eqs. (6)-(7); per-shell g, dt, N from per_shell[i]): blocks of check_every
 * steps, each captured once in a CUDA graph and replayed, followed by FP64
 * observables and the test |mu - mu_prev| < tol_dmu against the previous
 * check; a converged shell stops stepping while the others continue.  Stops
 * when every shell converged or after max_steps.  On return each state holds
 * its result; converged[i], steps[i] and obs[i] (any may be NULL) report each
 * shell.  GPE_ERR_NOT_CONVERGED if a shell did not converge,
 * GPE_ERR_NONFINITE if one produced NaN/Inf (it is stopped).  Synchronous. */
int gpe_batch_ground_state(gpe_batch *batch, const gpe_imag_params *per_shell,
                           double tol_dmu, int64_t check_every,
                           int64_t max_steps, int32_t *converged,
                           int64_t *steps, gpe_obs *obs, gpe_stream stream);

int gpe_batch_destroy(gpe_batch *batch);

/* ------------------------------------------------------------------ stages */
/* Multi-stage potential ramp (Sec. V).  The potential passes through the
 * precomputed potentials pots[0], ..., pots[n_pots-1]; stage i (i = 0 ..
 * n_pots-2) lasts durations[i] and interpolates linearly in time from
 * pots[i] to pots[i+1].  At the start of every stage the region of interest
 * is selected again and the wavefunction remapped onto it:
 *   mu_i   = Thomas-Fermi chemical potential of pots[i] for g and N (as
 *            gpe_tf_mu_*, Eq. (5)),
 *   cut_i  = cut_factor * max(mu_i, mu_{i+1})   (cut_factor = 5 in Sec. V),
 *   region = {V_i < cut_i} U {V_{i+1} < cut_i}, which holds every
 *            intermediate potential's region {V(s) < cut_i} (the union of
 *            the sublevel sets of a linear blend is that of its endpoints),
 * then the stage runs n = ceil(durations[i] / dt) equal real-time steps of
 * length durations[i] / n with V(t) = (1 - t/d) V_i + (t/d) V_{i+1}.  With
 * t_hold > 0 a hold in pots[n_pots-1] follows on the region
 * {V_last < cut_factor * mu_last}.
 *
 * psi0 is the initial state (complex, any grid over the box; it is read, not
 * changed).  The stage grids use *opts, or psi0's grid options when opts is
 * NULL.  A potential is analytic (analytic != NULL) or a dense box array
 * (V, V_dtype, V_on_device as in gpe_grid_create_dense); all of them must be
 * of one kind, and dense ones share V_dtype and V_on_device.
 *
 * On success *grid_out and *state_out receive the last stage's grid and the
 * final state (owned by the caller: destroy the state, then the grid).
 * report (may be NULL) receives n_pots - 1 entries, plus one for the hold.
 * Each stage's grids exist only while the stage runs; two grids and two
 * states are held at a time.  The remap drops the density outside the new
 * region (norm_kept reports what is left); there is no renormalisation.
 * Errors: GPE_ERR_ARG for bad arguments, else the failing call's code; on
 * error nothing is returned and everything made so far is freed.
 * Synchronous. */
typedef struct gpe_ramp_pot {
    const gpe_potential *analytic; /* non-NULL: analytic potential */
    const void *V;                 /* else: dense nx*ny*nz array */
    int32_t V_dtype, V_on_device;
} gpe_ramp_pot;

typedef struct gpe_stage_params {
    double g, N;          /* interaction and atom number (Thomas-Fermi mu) */
    double dt;            /* largest time step */
    double cut_factor;    /* region cutoff over max(mu_i, mu_{i+1}) */
    double t_hold;        /* hold in the last potential (0: none) */
    int32_t integrator;   /* GPE_RK4, GPE_RKHE3, GPE_RKCK */
    int32_t reserved;
} gpe_stage_params;

typedef struct gpe_stage_report {
    double mu_a, mu_b;     /* Thomas-Fermi mu of the stage's two potentials */
    double cut;            /* the cutoff used */
    int64_t n_active;      /* active cells of the stage's grid */
    int64_t steps;
    double dt;             /* step length used */
    double norm_kept;      /* sum |psi|^2 dV after the remap */
    double norm_end;       /* at the end of the stage */
    double regrid_s;       /* host seconds to build the grid, make the state
                              and remap (waited for when report is given) */
} gpe_stage_report;

int gpe_ramp_stages(const gpe_state *psi0, const gpe_ramp_pot *pots,
                    int n_pots, const double *durations,
                    const gpe_stage_params *p, const gpe_grid_opts *opts,
                    gpe_grid **grid_out, gpe_state **state_out,
                    gpe_stage_report *report, gpe_stream stream);

/* ------------------------------------------------------------------ adjoint */
/* Ramp gradient by the discrete adjoint of the RK4 step (not in the paper:
 * its ramps are optimised by a derivative-free search, Sec. V; here the
 * gradient is exact for the discrete RK4 map).
 *
 * gpe_ramp_forward runs nsteps real-time RK4 steps of a GPE_V_BLEND ramp from
 * the state's psi (as gpe_step_real, from time t0) and records a tape: a
 * checkpoint of psi every K steps, kept in device memory (ceil(nsteps/K)
 * copies of the state plus K more for the backward pass).  The state ends at
 * psi(T).  Asynchronous for the steps; returns the tape.
 *
 * gpe_ramp_backward computes L = 1 - |<target|psi(T)>|^2 (target: a state on
 * the same grid and type, e.g. the ground state of the final potential) and
 * dL/d knots[k] for k < n_knots, by recomputing each K-step segment from its
 * checkpoint and applying the transposed RK4 step in reverse (bulk in the
 * state's precision, gradient accumulated in FP64).  The tape can be reused
 * with other targets while the state still holds psi(T).  Synchronous. */
int gpe_ramp_forward(gpe_state *st, const gpe_real_params *p, int64_t nsteps,
                     double t0, int K, gpe_tape **out, gpe_stream stream);
int gpe_ramp_backward(gpe_tape *tape, const gpe_state *target,
                      double *grad_knots, double *loss, gpe_stream stream);
int gpe_tape_destroy(gpe_tape *tape);

/* ------------------------------------------------------------------ tuning */
enum { GPE_TUNE_REAL = 0, GPE_TUNE_IMAG = 1 };
typedef struct gpe_tune_result {
    int32_t bx, by, bz, sched, chunk, reserved;
    double cell_steps_per_s; /* active-cell-steps per second */
    double ms_per_step;
} gpe_tune_result;

/* Time every candidate layout (brick 8x8x8, 8x8x4, 8x4x4) and schedule
 * (staged; wavefront with 2-8 bricks per task; for GPE_TUNE_REAL also the RK4
 * stages fused in pairs, GPE_SCHED_PAIR, on 8x8x4 bricks) on the grid that
 * gpe_grid_create_analytic(box, pot, V_cut) builds, for `nsteps` real-time
 * (RK4) or imaginary-time steps of a state of type dtype (complex; real
 * types for imaginary time only), and return the fastest in *best (use its fields in gpe_grid_opts).  all (room for 8
 * entries, may be NULL) receives every timing and *n_all their number.
 * Results are cached per device, state type, step kind and size class
 * (n_active within a factor sqrt(2)); with all == NULL a cached answer is
 * returned without timing (*n_all = 0).  Synchronous; allocates temporary
 * grids. */
int gpe_autotune(const gpe_box *box, const gpe_potential *pot, double V_cut,
                 int dtype, int mode, int nsteps, gpe_tune_result *best,
                 gpe_tune_result *all, int *n_all, gpe_stream stream);

/* The brick shape for a batch of shells (gpe_batch_create; the batch kernels
 * run the staged schedule): for each candidate shape (8x8x8, 8x8x4, 8x4x4)
 * builds the n grids gpe_grid_create_analytic(boxes[i], pots[i], V_cuts[i])
 * makes, fills states of type dtype with a smooth test wavefunction, makes
 * the batch and times `nsteps` imaginary-time steps of all shells (g = 1,
 * N = 1, dt = 0.2 / (sum 2/h^2 + max V) per shell; the difference between
 * runs of one and two graph-replayed blocks of nsteps steps, so set-up and
 * copies cancel).  Returns the fastest in *best (cell_steps_per_s counts the
 * active cells of every shell), every timing in all (room for 3 entries, may
 * be NULL) and their number in *n_all.  Nothing is cached.  Synchronous;
 * allocates temporary grids, states and batches.  GPE_ERR_ARG for n < 1,
 * an unknown state type or nsteps < 1. */
int gpe_batch_autotune(const gpe_box *boxes, const gpe_potential *pots,
                       const double *V_cuts, int n, int dtype, int nsteps,
                       gpe_tune_result *best, gpe_tune_result *all,
                       int *n_all, gpe_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* GPE_H */
