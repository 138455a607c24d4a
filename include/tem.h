/*
 * tem.h -- C ABI of the GB300 step-off TEM forward model.
 *
 * The method (Boerner & Guettel, "Fast parallel transient electromagnetic
 * modeling using a uniform-in-time approximation to the exponential"):
 * the semi-discrete step-off field u(t) = exp(-t M^{-1} K) M^{-1} f
 * (Sec. 2.2, Eq. (expm)) is approximated at every channel t_k by one family
 * of rational functions with shared poles (Sec. 3.2, Eq. (ratfam)), so that
 *
 *     d_t b_z(r, t_k) ~= sum_i Re( c[i, k] q_r^T (K - xi_i M)^{-1} f )      (Eq. (rmj), (rmjQ))
 *
 * with one shifted solve per conjugate pair of poles, independent of the
 * number of channels.  K is the curl-curl operator and M the lumped
 * conductivity mass on a staggered (Yee) edge grid; f is a closed loop of
 * current; q_r reads d_t b_z at receiver r.
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  * Units: metres, seconds, S/m, amperes; mu0 = 4 pi 1e-7.  z points up.
 *  * Cells: nx x ny x nz with widths hx[nx], hy[ny], hz[nz] (> 0) from the
 *    corner `origin`.  Per-cell arrays are (nz, ny, nx), x fastest.
 *  * Complex numbers are interleaved (re, im) pairs of doubles.
 *  * Host pointers are owned by the caller and only read (or written, for
 *    outputs) during the call; the library keeps no reference to them.
 *  * `cuda_stream` is a cudaStream_t (NULL = legacy default stream).  Host
 *    outputs are complete when the call returns (it synchronises the stream).
 *  * Every entry point returns a status (TEM_OK = 0 on success) and never
 *    aborts the process; tem_status_string() names the code.  On an error
 *    other than TEM_ENOCONV no output is written.
 *  * Device memory comes from cudaMallocAsync on `cuda_stream`, or from the
 *    allocator installed with tem_set_allocator().
 *
 * Edge layout on the device (for tem_apply_operator): one complex vector is
 * 3 blocks (x-, y-, z-edges) of nx*ny*nz entries each, entry (c, i, j, k) at
 * c*nx*ny*nz + i + nx*(j + ny*k).  Entry (c, i, j, k) is the edge of
 * direction c leaving node (i, j, k).  Edges lying in the domain boundary
 * (n x e = 0, Eq. (bc)) hold 0; so do the padding entries (x-edges at
 * j = 0 or k = 0, and likewise for y and z).
 */
#ifndef TEM_H_
#define TEM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum {
  TEM_OK = 0,
  TEM_EINVAL = 1,      /* bad size, non-finite or non-positive value, geometry off the grid */
  TEM_ENOMEM = 2,      /* device allocation failed */
  TEM_ENOCONV = 3,     /* some shift reached max_iter; outputs are still written */
  TEM_EBREAKDOWN = 4,  /* COCG breakdown: (p, Ap) or (r, z) vanished or became non-finite */
  TEM_ETIMEOUT = 5,    /* a bounded wait ran out */
  TEM_ECUDA = 6,       /* a CUDA runtime call failed */
  TEM_EBUSY = 7        /* serving: the request has not finished yet */
};

/* ---- precision of the shifted solves ----------------------------------- */
enum {
  TEM_PREC_FP64 = 0,   /* FP64 COCG sweeps */
  TEM_PREC_MIXED = 1   /* FP32 COCG sweeps inside FP64 defect correction */
};

typedef struct tem_grid tem_grid;     /* opaque: device copy of the grid and conductivity */
typedef struct tem_state tem_state;   /* opaque: kept shifted solutions of one forward call */

/* Solver options.  Fill with tem_default_options() and then override. */
typedef struct tem_options {
  int32_t precision;     /* TEM_PREC_FP64 (default) or TEM_PREC_MIXED */
  int32_t max_iter;      /* bound on COCG iterations per shift (default 20000) */
  double tol;            /* stop when ||f - A_i x_i||_2 <= tol ||f||_2, FP64 residual (default 1e-12) */
  double inner_tol;      /* MIXED: relative residual reduction per FP32 inner solve (default 1e-1) */
  int32_t max_outer;     /* MIXED: bound on FP64 defect-correction steps (default 40) */
  int32_t check_every;   /* iterations between host-side convergence polls (default 32) */
  int32_t keep_state;    /* nonzero: keep the solutions for tem_adjoint (state_out must be non-NULL) */
  int32_t precond;       /* TEM_PRECOND_AUTO (default), TEM_PRECOND_JACOBI or TEM_PRECOND_NODAL */
  int32_t carry_direction; /* MIXED: nonzero (default 1): an FP64 outer step replaces the inner
                            residual by the true one and the inner COCG keeps its search
                            direction (residual replacement, once per inner_tol reduction);
                            0: every inner solve restarts from the true residual (plain defect
                            correction).  A solve that follows a stagnated inner solve restarts
                            either way */
} tem_options;

/* Preconditioner of the inner COCG sweeps. */
enum {
  TEM_PRECOND_AUTO = 0,    /* NODAL */
  TEM_PRECOND_JACOBI = 1,  /* z = D^{-1} r,  D = diag(K) - xi M */
  TEM_PRECOND_NODAL = 2    /* z = D^{-1} r + G D_n^{-1} G^T r: Jacobi plus a correction in the
                              nodal-gradient (near-null) space of K, D_n = -xi diag(G^T M G).
                              Relies on G^T b = 0 for the right-hand side b (true for closed
                              loop sources and for receiver-adjoint sources) */
};

/* Default options (see the field comments). */
void tem_default_options(tem_options* opt);

/* Name of a status code (static string). */
const char* tem_status_string(int status);

/* Library version string. */
const char* tem_version(void);

/* Text of the last CUDA error seen by this thread's calls (empty if none). */
const char* tem_last_error(void);

/*
 * Install the device allocator used for every buffer the library creates.
 * alloc(bytes, stream, ctx) returns a 256-byte aligned device pointer or NULL;
 * release(ptr, bytes, stream, ctx) frees it.  Passing NULL for both restores
 * cudaMallocAsync / cudaFreeAsync.  Not thread-safe with calls in flight.
 */
typedef void* (*tem_alloc_fn)(size_t bytes, void* cuda_stream, void* ctx);
typedef void (*tem_free_fn)(void* ptr, size_t bytes, void* cuda_stream, void* ctx);
int tem_set_allocator(tem_alloc_fn alloc, tem_free_fn release, void* ctx);

/*
 * Build the device-side grid (Sec. 2.2: the discretisation of Eq. (pde)-(source)).
 *   hx, hy, hz : cell widths, lengths nx, ny, nz >= 2, all finite and > 0.
 *   origin     : 3 doubles, coordinates of node (0, 0, 0).
 *   sigma      : nx*ny*nz cell conductivities (S/m), finite and > 0.
 *   out        : receives the handle; release with tem_grid_destroy().
 * Computes the lumped edge mass M_e = sum over the 4 cells containing e of
 * sigma_c V_c / 4 (FP64 and an FP32 copy) and the 1-D face factors of K.
 * Errors: TEM_EINVAL for bad sizes or values, TEM_ENOMEM, TEM_ECUDA.
 */
int tem_build_grid(const double* hx, int64_t nx, const double* hy, int64_t ny,
                   const double* hz, int64_t nz, const double* origin,
                   const double* sigma, void* cuda_stream, tem_grid** out);

/* Replace the conductivity of an existing grid (same sizes and rules as tem_build_grid).
   A state kept by an earlier tem_forward on this grid belongs to the old conductivity: after
   this call, tem_adjoint and tem_jvp on that state return TEM_EINVAL (run the forward again). */
int tem_grid_set_sigma(tem_grid* grid, const double* sigma, void* cuda_stream);

/* Grid sizes: dims[0..2] = nx, ny, nz; returns TEM_EINVAL on NULL. */
int tem_grid_dims(const tem_grid* grid, int64_t* dims);

int tem_grid_destroy(tem_grid* grid);

/*
 * Shared poles and per-channel weights (Sec. 3.2, Eq. (ratfam)-(rkfit), (rmj)).
 *   t        : K >= 1 channel times (s), finite, > 0, strictly increasing.
 *   degree   : number of poles m-hat, 1 <= degree <= 64.
 *   weights  : K positive weights w_k of the fit objective, or NULL for all ones.
 *   xi       : out, 2*s doubles: the shifts (one pole of each conjugate pair,
 *              with Im > 0, then the real poles), physical units (1/s).
 *   c        : out, 2*s*K doubles, row-major [s][K]: c = 2 alpha for a pair,
 *              alpha for a real pole, so that exp(-t_k lam) ~= sum_i Re(c[i,k] / (lam - xi_i)).
 *              Caller allocates both with s = degree (an upper bound).
 *   s_out    : out, the number of shifts s = ceil(degree / 2) for all-complex families.
 *   uniform_err_out : out (may be NULL), Eq. (uniform_error): max_k w_k max_{x>=0} |e^{-t_k x} - r^[k](x)|
 *              on a fine sample of [0, inf), in the normalised variable (t / t_max).
 * The fit is the RKFIT pole relocation on a diagonal surrogate (times
 * normalised by t_max), in FP64 on the host.  Errors: TEM_EINVAL.
 */
int tem_poles_residues(const double* t, int64_t K, int64_t degree, const double* weights,
                       double* xi, double* c, int64_t* s_out, double* uniform_err_out);

/*
 * One step-off forward model (Eq. (rmjQ)):
 *   d[r, k] = sum_i Re( c[i, k] q_r^T (K - xi_i M)^{-1} f ).
 *   grid       : from tem_build_grid.
 *   loop_xy    : n_vertices (x, y) pairs of a closed axis-aligned polygon
 *                whose vertices are grid nodes, on the node plane z = z_loop;
 *                counter-clockwise seen from +z gives a +z moment.
 *   current    : loop current I (A).
 *   rx_xyz     : n_rx receivers (x, y, z) inside the grid; z snaps to the
 *                nearest node plane; d_t b_z is interpolated bilinearly
 *                between z-face centres.  1 <= n_rx <= 4096.
 *   xi, c, s, K: as returned by tem_poles_residues (1 <= s <= 64).
 *   opt        : solver options (NULL = defaults).
 *   dbzdt_out  : host, n_rx*K doubles, row-major [n_rx][K], d_t b_z in T/s.
 *   state_out  : if opt->keep_state, receives the kept solutions for
 *                tem_adjoint (release with tem_state_destroy); else may be NULL.
 * Returns TEM_ENOCONV (output written) if a shift hit max_iter,
 * TEM_EBREAKDOWN on a COCG breakdown, TEM_EINVAL on bad geometry, TEM_ETIMEOUT if a bounded
 * device-side wait of the FP32 stencil ran out (its slot stops; nothing hangs).
 */
int tem_forward(const tem_grid* grid, const double* loop_xy, int64_t n_vertices,
                double z_loop, double current, const double* rx_xyz, int64_t n_rx,
                const double* xi, const double* c, int64_t s, int64_t K,
                const tem_options* opt, void* cuda_stream, double* dbzdt_out,
                tem_state** state_out);

/*
 * Several loop sources on one grid in one batched solve (the block source f of Sec. 4, "Using
 * multiple sources"): source j is the closed polygon loops_xy[2 * vert_off[j] .. 2 * vert_off[j+1])
 * (x, y pairs, at least 3 vertices) at height z_loops[j] carrying currents[j]; all sources share
 * the receivers rx_xyz, the shifts xi and the channel weights c (same meaning as tem_forward).
 * The n_src * s shifted systems advance together, one launch per pass for all of them; each
 * system's arithmetic depends only on its own data, so the result equals n_src separate
 * tem_forward calls bit for bit.  dbzdt_out (host, caller-owned) holds n_src * n_rx * K
 * doubles, source-major, each source's block laid out like tem_forward's output.
 * 1 <= n_src <= 1024; opt->keep_state must be 0 (no state is kept).  Returns TEM_EINVAL for
 * bad sizes, loops or receivers (before any device work), TEM_ENOCONV (output written),
 * TEM_EBREAKDOWN, TEM_ENOMEM or TEM_ECUDA.
 */
int tem_forward_sources(const tem_grid* grid, const double* loops_xy, const int64_t* vert_off, int64_t n_src,
                        const double* z_loops, const double* currents, const double* rx_xyz, int64_t n_rx,
                        const double* xi, const double* c, int64_t s, int64_t K, const tem_options* opt,
                        void* cuda_stream, double* dbzdt_out);

/*
 * The single-time best-approximation baseline (Sec. 3.1, Eq. (rba)), the comparison method of the
 * paper: one rational approximant r(x) = sum_i Re(c_i / (x - xi_i)) ~= exp(-x) on x >= 0 (xi, c as
 * returned by tem_poles_residues for the single time t = 1, so s shifts and one channel) is
 * evaluated at every channel t_k separately:
 *   d[r, k] = sum_i Re( c_i q_r^T (t_k K - xi_i M)^{-1} f )
 *           = sum_i Re( (c_i / t_k) q_r^T (K - (xi_i / t_k) M)^{-1} f ),
 * i.e. K * s shifted solves instead of the s of tem_forward's shared poles; they run through the
 * same batched solver, 64 shifts at a time.  t: K channel times (s), finite and > 0.  Other
 * arguments, the output layout and the statuses as for tem_forward (opt->keep_state is ignored).
 * solves_out (may be NULL) receives K * s.
 */
int tem_forward_single_time(const tem_grid* grid, const double* loop_xy, int64_t n_vertices, double z_loop,
                            double current, const double* rx_xyz, int64_t n_rx, const double* t, int64_t K,
                            const double* xi, const double* c, int64_t s, const tem_options* opt,
                            void* cuda_stream, double* dbzdt_out, int64_t* solves_out);

/*
 * Per-shift diagnostics of the last forward (or adjoint) solve kept in `state`:
 *   iters[s]   : COCG iterations (inner FP32 iterations summed, for MIXED),
 *   relres[s]  : final FP64 relative residual ||f - A_i x_i|| / ||f||.
 * Either pointer may be NULL.
 */
int tem_state_stats(const tem_state* state, int32_t* iters, double* relres);

/*
 * Copy the FP64 solution x_i = (K - xi_i M)^{-1} f of shift i (the solves of Eq. (rmj)) kept in
 * `state` to host memory.  x_out (caller-owned) holds 2 * 3 * nx * ny * nz doubles, (re, im)
 * interleaved, in the edge layout of the library: entry (c, i, j, k) at
 * c * nx*ny*nz + i + nx * (j + ny * k) is the edge of direction c leaving node (i, j, k);
 * boundary and padding entries are 0.  Synchronises `cuda_stream`.
 * TEM_EINVAL for a NULL pointer or i outside [0, s).
 */
int tem_state_solution(const tem_state* state, int64_t i, void* cuda_stream, double* x_out);

/*
 * Time snapshots of the field, the columns of S R in Sec. 3.2: for the channels
 * k = k0 .. k0+nk-1 writes u_k[e] = sum_i Re(c[i, k] x_i[e]) (Eq. (rmj) on every edge: the
 * rational approximation of exp(-t_k M^{-1} K) M^{-1} f) to u_dev, caller-owned DEVICE memory of
 * nk * 3 * nx*ny*nz doubles, channel-major, each channel in the edge layout of
 * tem_state_solution.  Enqueued on cuda_stream, not synchronised.  TEM_EINVAL for NULL
 * pointers or a channel range outside [0, K).
 */
int tem_state_fields(const tem_state* state, int64_t k0, int64_t nk, void* cuda_stream, void* u_dev);

/*
 * Adjoint gradient (Sec. 4): given g = dphi/dd (host, n_rx*K doubles laid
 * out like dbzdt_out), writes grad[c] = dphi/dlog sigma_c for every cell
 * (host, nx*ny*nz doubles):
 *   beta[i, r] = sum_k c[i, k] g[r, k],   w_i = sum_r beta[i, r] q_r,
 *   lambda_i = (K - xi_i M)^{-1} w_i      (A_i is complex symmetric),
 *   grad[c] = sum_i Re( xi_i sum_{e in c} (sigma_c V_c / 4) lambda_i[e] x_i[e] ).
 * The adjoint solves use the precision and tolerances of the forward call.
 * Returns TEM_ENOCONV (gradient written) if an adjoint solve hit max_iter, TEM_EINVAL if the
 * grid's conductivity was replaced (tem_grid_set_sigma) after the forward call.
 */
int tem_adjoint(tem_state* state, const double* dphi_dd, void* cuda_stream, double* grad_logsigma_out);

/*
 * Linearised forward, the Jacobian-vector product of Sec. 4: for a direction dm in
 * log sigma (host, nx*ny*nz doubles, one per cell) writes dd = J dm (host, n_rx*K doubles laid
 * out like dbzdt_out):
 *   dM_e = sum_{cells c around e} sigma_c dm_c V_c / 4,     b_i = xi_i dM x_i,
 *   dx_i = (K - xi_i M)^{-1} b_i,                          dd[r, k] = sum_i Re(c[i, k] q_r^T dx_i),
 * with x_i the forward solutions kept in `state` (one batched solve of the s shifts, the
 * precision and tolerances of the forward call; the nodal preconditioner adds the
 * divergence of b_i, which is not zero here).  J^T is tem_adjoint: the two satisfy
 * <g, J dm> = <tem_adjoint(g), dm>.  A zero direction returns zeros without a solve.
 * Returns TEM_EINVAL for NULL pointers, a non-finite entry of dm or a conductivity replaced
 * after the forward call, TEM_ENOCONV (output written) if a solve hit max_iter.
 */
int tem_jvp(tem_state* state, const double* dlogsigma, void* cuda_stream, double* ddbzdt_out);

int tem_state_destroy(tem_state* state);

/*
 * Apply the shifted operator to s device vectors (the hot stencil, Sec. 2.2 K and M):
 *   q[i] = (K - xi_i M) p[i],  i < s.
 *   p_dev, q_dev : device, s complex vectors in the edge layout above, each
 *                  3*nx*ny*nz complex entries; p's boundary entries must be 0,
 *                  q's are written as 0.  FP64 (double2) if precision is
 *                  TEM_PREC_FP64, FP32 (float2) if TEM_PREC_MIXED.
 *   xi           : host, 2*s doubles.
 * Enqueued on cuda_stream; returns without synchronising.
 */
int tem_apply_operator(const tem_grid* grid, const double* xi, int64_t s,
                       const void* p_dev, void* q_dev, int32_t precision, void* cuda_stream);

/* ---- serving: continuous batching of forward models -------------------------
 *
 * A server owns one CUDA stream's worth of device work.  Requests (each a whole
 * forward model: grid, conductivity, loop, receivers, shifts, weights) are queued
 * by tem_server_submit, admitted in arrival order when enough slots (one per
 * shift) are free and their device footprint fits the HBM budget, and then
 * advanced together: every tem_server_step launches the stencil, update and
 * nodal passes once per COCG iteration over the shifts of all admitted requests
 * at once (plus the FP64 residual passes of shifts whose inner solve ended).
 * A request that arrives while others run is admitted at the next step that has
 * room; its Krylov state stays on the device until it finishes.  Each shift's
 * arithmetic (its tiling and the order of its reductions) depends only on its own
 * grid, so a request's result is bitwise the same alone and in any mix.
 * Not thread-safe: one host thread drives a server.
 */
typedef struct tem_server tem_server;

typedef struct tem_server_options {
  int64_t hbm_budget_bytes;  /* admit while the footprints of running requests fit (default: 80% of free memory) */
  int32_t max_slots;         /* shifted systems in flight at once (default 128, at most 1024) */
  int32_t iters_per_step;    /* COCG iterations per tem_server_step (default 32) */
  tem_options solver;        /* precision, tolerances, preconditioner (keep_state is ignored) */
} tem_server_options;

typedef struct tem_request_stats {
  double submit_s, admit_s, done_s;  /* host steady-clock times (s) */
  int64_t footprint_bytes;           /* device bytes the request held while running */
  int32_t status;                    /* TEM_OK, TEM_ENOCONV, TEM_EBREAKDOWN or TEM_ETIMEOUT */
  int32_t max_iters;                 /* largest per-shift COCG iteration count */
} tem_request_stats;

void tem_server_default_options(tem_server_options* opt);
int tem_server_create(const tem_server_options* opt, void* cuda_stream, tem_server** out);
/* Queue one forward model (arguments as for tem_build_grid and tem_forward; all are copied).
   Errors: TEM_EINVAL for bad input (checked now, on the host). */
int tem_server_submit(tem_server* srv, const double* hx, int64_t nx, const double* hy, int64_t ny,
                      const double* hz, int64_t nz, const double* origin, const double* sigma,
                      const double* loop_xy, int64_t n_vertices, double z_loop, double current,
                      const double* rx_xyz, int64_t n_rx, const double* xi, const double* c, int64_t s,
                      int64_t K, int64_t* ticket_out);
/* One scheduling round: admit what fits, run iters_per_step iterations for every admitted
   request, finish the requests whose shifts have all converged.  Returns after the round. */
int tem_server_step(tem_server* srv);
/* TEM_EBUSY while the request is queued or running; otherwise its status, with
   dbzdt_out (n_rx*K doubles) and stats written once (the ticket is then released). */
int tem_server_poll(tem_server* srv, int64_t ticket, double* dbzdt_out, tem_request_stats* stats);
int tem_server_counts(const tem_server* srv, int64_t* queued, int64_t* running, int64_t* finished);
int tem_server_destroy(tem_server* srv);

/*
 * tem_apply_operator without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that may not allocate device memory, such as a
 * host framework that owns all device memory through its own pool, or a latency-bound
 * loop that must not risk the device-wide synchronisation cudaMalloc/cudaFree can cause.
 * Same arguments, layout and result as tem_apply_operator (q[i] = (K - xi_i M) p[i]),
 * with these differences:
 *   - s <= 64 (TEM_EINVAL otherwise); the shifts are copied into one fixed 1 KB array
 *     in device memory that the library defines statically, instead of a per-call buffer;
 *   - the grid's device must be the current device (TEM_EINVAL otherwise);
 *   - the first call on a device looks up that array's device address once
 *     (cudaGetSymbolAddress) and keeps it for the life of the process: it assumes the
 *     runtime's primary context of that device and no cudaDeviceReset in between; make that
 *     first call before any stream capture;
 *   - every call shares the array and leaves its shifts there; calls whose work
 *     overlaps on the GPU (for example on two streams at once) race on it.
 * Enqueued on cuda_stream; returns without synchronising.  Allocates nothing.
 */
int tem_apply_operator_noalloc(const tem_grid* grid, const double* xi, int64_t s,
                               const void* p_dev, void* q_dev, int32_t precision, void* cuda_stream);

/*
 * Number of CUDA kernels this library has launched in this process so far
 * (monotone; for launch accounting around a timed region).
 */
int64_t tem_launch_count(void);

/*
 * Per-kernel timing of the solver's passes (measurement support; no paper
 * counterpart beyond the solves of Eq. (rmj)).  Sets up the batched solve of
 * tem_forward for `s` shifts (same loop source; precision and preconditioner as given), runs one
 * FP64 residual pass and then `n_iter` COCG iterations with CUDA events around
 * every launch on `cuda_stream`, and writes the average duration in ms of
 *   ms_out[0] : the stencil pass  (a, b <- z parts + beta a, b; q <- A (a + G b); G^T M p; (p, q)),
 *   ms_out[1] : the update pass   (x, x_n, r, w = D^-1 r, G^T M d, psi; (r, z), ||r||),
 *   ms_out[2] : the FP64 residual pass,
 *   ms_out[3] : not a time: the CTAs per SM the FP32 stencil kernel keeps resident
 *               (0 for FP64),
 * and units_out[0] = interior edges x shifts processed per launch.
 * Slots that converge before n_iter stop being timed; use n_iter small enough.
 */
int tem_profile_passes(const tem_grid* grid, const double* loop_xy, int64_t n_vertices, double z_loop,
                       double current, const double* xi, int64_t s, int32_t precision, int32_t precond,
                       int32_t n_iter,
                       void* cuda_stream, double* ms_out, double* units_out);

#ifdef __cplusplus
}
#endif

#endif /* TEM_H_ */
