/*
 * tsu.h -- C ABI of libtsu, a GB300 (sm_103a) explicit leapfrog stepper for the
 * regularised 2D tsunami wave equation of
 *   "Tsunami propagation for singular topographies" (arXiv:2005.11931):
 *
 *     u_tt = d_x(h_x d_x u) + d_y(h_y d_y u)        Sec. 2, eq. (2.1) (vector depth)
 *     u(0) = u0, u_t(0) = u1                        Cauchy data, eq. (2.1)
 *     u = 0 on the edges of the box [0,1]^2          Sec. 3.3 (2D boundary value problem)
 *     h_eps = h * psi_eps, psi_eps = eps^-d psi(./eps)  Sec. 2.1 (regularisation), Sec. 3.1
 *
 * Discretisation (the library's definition of every result):
 *   grid     x_i = i dx, y_j = j dy, i < nx, j < ny (boundary nodes included), Sec. 3.3 grid omega.
 *   faces    hx[j][i] = h_eps(x_i + dx/2, y_j), i <= nx-2;  hy[j][i] = h_eps(x_i, y_j + dy/2), j <= ny-2.
 *   operator B u = cx [hx_ij (u_i+1 - u_i) - hx_i-1,j (u_i - u_i-1)]
 *                + cy [hy_ij (u_j+1 - u_j) - hy_i,j-1 (u_j - u_j-1)],  cx = tau^2/dx^2, cy = tau^2/dy^2
 *            (B = tau^2 L_h, the conservative 5-point form of eq. (2.1)'s spatial part).
 *   start    u^1 = u^0 + tau u1 + B u^0 / 2              (Taylor start; the start counts as step 1)
 *   leapfrog u^{n+1} = 2 u^n - u^{n-1} + B u^n            (interior nodes; edges stay 0)
 *   energy   E^{n+1/2} = dxdy/(2 tau^2) sum_nodes [(u^{n+1}-u^n)^2 - (B u^{n+1}) u^n],
 *            the leapfrog analogue of the conservation law (CL-01) in Theorem 2.1; it equals
 *            1/2 sum ((u^{n+1}-u^n)/tau)^2 dxdy + 1/2 sum_faces h (D u^{n+1})(D u^n) dxdy.
 *
 * Memory layout: every field is row-major, x fastest, a[j*ld + i], ny rows of ld elements,
 * ld >= nx and ld a multiple of 4; every pointer 16-byte aligned.  Entries with i >= nx
 * (padding) are read and written as 0; the caller allocates them.
 *
 * Ownership: the caller owns every buffer (host or device, as stated per argument).  The
 * library keeps no pointer after a call returns and allocates no device memory: scratch is
 * the caller's workspace (sizes from tsu_*_workspace).  Work is enqueued on the caller's
 * stream (a cudaStream_t passed as void*; NULL is the legacy default stream) and is
 * asynchronous unless an argument says the call synchronises.
 *
 * Errors: every entry point returns a tsu_status.  On failure nothing is enqueued (argument
 * errors) or the CUDA error is reported (TSU_ECUDA); tsu_last_error() gives a message for the
 * calling thread.
 */
#ifndef TSU_H
#define TSU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TSU_OK = 0,
  TSU_EINVAL = 1,   /* null pointer, nx or ny < 3, ld < nx, ld % 4 != 0, misaligned pointer, bad enum */
  TSU_ECFL = 2,     /* tau^2 (hx_max/dx^2 + hy_max/dy^2) > 1: outside the leapfrog stability bound */
  TSU_ENONPOS = 3,  /* min face depth <= 0: the positivity 0 < c0 <= h_j of Sec. 2 fails */
  TSU_ENOMEM = 4,   /* caller workspace smaller than tsu_*_workspace reports */
  TSU_ECUDA = 5,    /* a CUDA runtime error (message in tsu_last_error) */
  TSU_ETIMEOUT = 6  /* a bounded device-side wait expired */
} tsu_status;

enum { TSU_F32 = 0, TSU_F64 = 1 };                      /* element type of u, hx, hy, traces */
enum { TSU_FORM_STANDARD = 0, TSU_FORM_INCREMENT = 1 }; /* see tsu_state */
enum { TSU_LINE_X = 0, TSU_LINE_Y = 1, TSU_POINT = 2, TSU_STEP_X = 3, TSU_STEP_Y = 4 };
enum { TSU_GAUSS = 0, TSU_FRIEDRICHS = 1 };

/* Unit-box grid: nx x ny nodes including the boundary; dx = 1/(nx-1), dy = 1/(ny-1) are
 * passed explicitly so callers may scale the box. */
typedef struct {
  int32_t nx, ny;
  int64_t ld; /* row pitch in elements */
  double dx, dy;
} tsu_grid;

/* One singularity of the depth (Sec. 3.1, Cases 1-3; Sec. 3.3):
 *   TSU_LINE_X  amp * phi_eps(x - cx)^power      (a line delta across the box, h varies in x)
 *   TSU_LINE_Y  amp * phi_eps(y - cy)^power
 *   TSU_POINT   amp * phi2_eps(|(x,y) - (cx,cy)|)^power   (2D mollifier, eps^-2 scaling)
 *   TSU_STEP_X  amp * Phi_eps(cx - x)             (mollified jump: amp for x < cx, 0 after)
 *   TSU_STEP_Y  amp * Phi_eps(cy - y)
 * power 1 is the delta, power 2 the delta^2 of Case 3 (phi_eps^2). */
typedef struct {
  int32_t kind, power;
  double amp, cx, cy;
} tsu_sing;

/* Depth h_eps = background + sum of singularities, regularised at width eps with
 *   TSU_GAUSS       phi_eps(s) = exp(-s^2/eps^2)/(eps sqrt(pi)), phi2_eps(r) = exp(-r^2/eps^2)/(pi eps^2)
 *   TSU_FRIEDRICHS  phi_eps(s) = c1/eps bump(s/eps), phi2_eps(r) = c2/eps^2 bump(r/eps),
 *                   bump(t) = exp(1/(t^2-1)) on |t| < 1 (Sec. 3.1, c1 ~ 2.2523). */
typedef struct {
  double background, eps;
  int32_t mollifier, nsing;
  const tsu_sing* sing; /* host array [nsing] */
} tsu_depth;

/* The medium as the steppers see it: device face arrays (element type = dtype) and the face
 * extrema returned by tsu_make_depth (ext = {min hx, max hx, min hy, max hy}).  Every stepper
 * checks them before it enqueues anything:
 *   - positivity (Sec. 2, 0 < c0 <= h_j): each face family has 0 < min <= max, or is identically
 *     zero (min = max = 0: the equation then decouples into 1D problems along the other
 *     direction, the paper's 1D setting), and not both families are zero; otherwise TSU_ENONPOS;
 *   - the leapfrog bound tau^2 (hx_max/dx^2 + hy_max/dy^2) <= 1; otherwise TSU_ECFL.
 * The extrema are the caller's statement about the arrays; the kernels do not re-check them. */
typedef struct {
  const void* hx;
  const void* hy;
  double hx_max, hy_max;
  double hx_min, hy_min;
} tsu_medium;

/* Time-stepping state (device buffers of ny*ld elements, owned by the caller).
 *   buf[cur] = u^n;  buf[aux] = u^{n-1} (TSU_FORM_STANDARD) or v^n = u^n - u^{n-1}
 *   (TSU_FORM_INCREMENT); the other buffers are scratch the steppers write into.
 *   TSU_FORM_STANDARD : a plain step writes u^{n+1} over u^{n-1} (needs nbuf >= 2).
 *   TSU_FORM_INCREMENT: a plain step writes v^{n+1} = v^n + B u^n in place and u^{n+1} = u^n + v^{n+1}
 *                       into a scratch buffer (nbuf >= 3).  Same scheme, rounded differently: it
 *                       keeps FP32 fields accurate when the per-step change is far below one ulp of u.
 *   FP32 fields in TSU_FORM_STANDARD lose part of every update whose size is below one ulp of u,
 *   and that error grows with the step count: over thousands of small steps they do NOT stay
 *   within 1e-5 relative L2 of the FP64 solution (a 400-step run of a ragged grid is already at
 *   ~3e-5).  Use TSU_FORM_INCREMENT for long FP32 runs; the standard form is exact in FP64 and for
 *   data where each update is representable (d'Alembert at Courant number 1).
 *   The temporally blocked kernel writes both output levels into scratch buffers (nbuf = 4).
 * step = n.  cur, aux and step are updated on the host when work is enqueued.  tsu_init fills
 * every provided buffer (scratch buffers with zeros). */
typedef struct {
  void* buf[4];
  int32_t nbuf;
  int32_t form;
  int32_t cur, aux;
  int64_t step;
} tsu_state;

/* Optional outputs and tuning of tsu_step_n (pass NULL for none / defaults).  For a call that
 * starts at step s and makes nsteps steps, step k (k = 0..nsteps-1) reads the pair (u^{s+k-1},
 * u^{s+k}) and produces u^{s+k+1}; on the way it records
 *   energy[k]          = E^{s+k-1/2}                      (device double [nsteps])
 *   traces[k*nrec + r] = u^{s+k}[rec_idx[r]]              (device, element type = dtype)
 * and, when (s+k-1) % ckpt_every == 0, copies the state (both fields of the form) into slot
 * (s+k-1)/ckpt_every of ckpt (device, [slots][2][ny][ld]); slots beyond ckpt_slots are skipped.
 * The final pair's energy and traces come from tsu_observe. */
typedef struct {
  double* energy;
  int32_t nrec;
  const int64_t* rec_idx; /* device [nrec], flat node indices j*ld + i */
  void* traces;
  void* ckpt;
  int64_t ckpt_every, ckpt_slots;
  int32_t kernel;   /* 0 auto, 1 register-streaming (one step per pass), 2 warp-blocked (tdepth =
                       2 or 4 steps per pass, default 4), 3 CTA-blocked (tdepth = 4 or 8, default 8);
                       2 and 3 need FP32, nbuf = 4 and a workspace; 2 records up to 2048
                       receivers and takes checkpoints when ckpt_every is a multiple of tdepth and
                       the call starts at step 1 + j tdepth; 3 takes neither; 4 runs kernel 2's
                       passes (tdepth 4, increment form, no traces or checkpoints) all in one
                       persistent launch, a tile's next pass starting once the tiles
                       around it finished the current one (its waits are bounded: TSU_ETIMEOUT
                       through tsu_sync_status); auto picks kernel 4 where it can run and its tiles
                       number between half and 6 times the device's resident warps (FP32 grids
                       of about 2K to 12K per side), else kernel 2 (tdepth 4) whenever it can.  All
                       kernels round every operation the same way, so the FP32 states do not
                       depend on the choice */
  int32_t rows;     /* rows per CTA (kernels 1, 3) or per warp tile (kernels 2, 4); 0 = auto */
  int32_t tdepth;   /* steps per pass of kernels 2 and 3 (0 = default); leftover steps run one per pass */
  int32_t reserved; /* 0.  Bits 0 and 1 are test hooks of the failure detection: with bit 0
                       kernel 3 never issues one row copy, with bit 1 kernel 4 never reports
                       tile 0 done; their bounded waits (20 ms) expire and tsu_sync_status
                       reports TSU_ETIMEOUT; outputs of that call are invalid. */
} tsu_step_opts;

/* Library version (major*10000 + minor*100 + patch). */
int tsu_version(void);

/* Message describing the last failure on the calling thread ("" if none). */
const char* tsu_last_error(void);

/* Face coefficients of the regularised depth (Sec. 2.1 h_eps = h * psi_eps; Sec. 3.1 mollifier).
 *   g        grid; d  depth descriptor (host); dtype TSU_F32/TSU_F64 of hx, hy.
 *   hx, hy   device [ny][ld], written completely (unused faces and padding = 0).
 *   ext_dev  device double[4] receiving {min hx, max hx, min hy, max hy} over the defined faces.
 *   ext_host host double[4] or NULL; when given, the call synchronises the stream, copies ext,
 *            and returns TSU_ENONPOS if a minimum is <= 0.
 * The depth is evaluated in FP64 and rounded once to dtype. */
int tsu_make_depth(const tsu_grid* g, const tsu_depth* d, int dtype, void* hx, void* hy,
                   double* ext_dev, double* ext_host, void* stream);

/* d h_eps / d eps: the derivative of the regularised depth in its width (Sec. 2.1, h_eps = h *
 * psi_eps with psi_eps(s) = eps^-d psi(s/eps), so d/deps psi_eps = -eps^-(d+1) (d psi + t psi'(t)),
 * t = s/eps; for a mollified step S = int^{s/eps} psi, dS/deps = -(t/eps) psi(t)), sampled at
 * the faces exactly like tsu_make_depth's hx, hy (same layout, element type dtype, entries
 * outside the faces 0).  Evaluated in FP64.  Asynchronous.  Errors: TSU_EINVAL, TSU_ECUDA. */
int tsu_depth_eps_derivative(const tsu_grid* g, const tsu_depth* d, int dtype, void* dhx, void* dhy, void* stream);

/* Bytes of device workspace (16-byte aligned) of the reductions below. */
size_t tsu_reduce_workspace(void);

/* dJ/deps = sum over faces of g_hx dhx/deps + g_hy dhy/deps: chains face gradients (device double
 * [ny][ld], e.g. tsu_adjoint's g_hx, g_hy) through the regularised depth, without storing the
 * derivative fields.  Deterministic FP64 sum (fixed grid, fixed order) into out_dev[0] (device
 * double).  Asynchronous.  Errors: TSU_EINVAL, TSU_ENOMEM (workspace), TSU_ECUDA. */
int tsu_depth_eps_gradient(const tsu_grid* g, const tsu_depth* d, const double* g_hx, const double* g_hy,
                           double* out_dev, void* ws, size_t ws_bytes, void* stream);

/* How far apart two fields are (the eps-family comparisons of Sec. 3.2): out_dev[0] = sum (a - b)^2,
 * out_dev[1] = sum b^2 over the nodes i < nx of two device fields of element type dtype.
 * Deterministic FP64 sums.  Asynchronous.  Errors: TSU_EINVAL, TSU_ENOMEM, TSU_ECUDA. */
int tsu_diff_norms(const tsu_grid* g, int dtype, const void* a, const void* b, double* out_dev, void* ws,
                   size_t ws_bytes, void* stream);

/* Largest tau allowed by the leapfrog bound tau^2 (hx_max/dx^2 + hy_max/dy^2) <= 1, times cfl
 * (0 < cfl <= 1).  Host only.  Returns 0 on bad input. */
double tsu_tau_for(const tsu_grid* g, double hx_max, double hy_max, double cfl);

/* The time step of the workloads: tau = courant * min(dx, dy) / sqrt(max(hx_max, hy_max)), a
 * Courant number relative to the fastest wave speed sqrt(h) over the sampled faces (the 2D runs
 * of Sec. 3.3 take a fixed Courant number; the workloads here use 0.4).  Inside the leapfrog
 * bound for courant <= 1/sqrt(2); the implicit comparator below also takes larger ones.  Host
 * only.  Returns 0 on bad input (courant not positive and finite, no positive face maximum). */
double tsu_tau_courant(const tsu_grid* g, const tsu_medium* m, double courant);

/* Cauchy data to the first two time levels (eq. (2.1) initial conditions; Taylor start above).
 *   u0       device [ny][ld] displacement (boundary values ignored: taken as 0).
 *   u1       device [ny][ld] velocity, or NULL for u1 = 0.
 *   st       st->buf[0..nbuf-1] device buffers, st->nbuf and st->form are read.  On return
 *            st->step = 1 and cur/aux are set (standard: buf[0] = u^0, buf[1] = u^1;
 *            increment: buf[0] = u^1, buf[1] = v^1 = tau u1 + B u^0 / 2).
 * Errors: TSU_EINVAL, TSU_ENONPOS (the medium's extrema, see tsu_medium), TSU_ECFL. */
int tsu_init(const tsu_grid* g, int dtype, double tau, const tsu_medium* m, const void* u0,
             const void* u1, tsu_state* st, void* stream);

/* Bytes of device workspace tsu_step_n and tsu_observe need: a status word, the energy partial
 * sums and, for the warp-blocked pass, a table of each tile's receivers (rebuilt by every call
 * that records traces). */
int tsu_step_workspace(const tsu_grid* g, int dtype, size_t* bytes);

/* Advance the state by nsteps leapfrog steps (the hot path; scheme above).
 *   opts  NULL or tsu_step_opts (outputs, tuning).  ws/ws_bytes: device workspace of
 *         tsu_step_workspace bytes (or NULL), zero-filled by the caller before its first use;
 *         needed for the energy and the temporally blocked kernel.
 * Errors: TSU_EINVAL, TSU_ENONPOS, TSU_ECFL, TSU_ENOMEM, TSU_ECUDA. */
int tsu_step_n(const tsu_grid* g, int dtype, double tau, const tsu_medium* m, tsu_state* st,
               int64_t nsteps, const tsu_step_opts* opts, void* ws, size_t ws_bytes, void* stream);

/* Number of checkpoint slots a forward run of nsteps steps (Taylor start included) fills when
 * tsu_step_n is given ckpt_every: states m = 1, 1 + every, ... <= nsteps - 1.  Host only. */
int64_t tsu_ckpt_slots(int64_t nsteps, int64_t ckpt_every);

/* Bytes of device workspace tsu_adjoint needs for a forward run of this form with nrec receivers:
 * 2 ckpt_every + 10 fields of dtype (four multiplier fields and two recompute segments of
 * ckpt_every + 3 fields), two FP32 gradient accumulators for FP32 fields and receiver tables. */
int tsu_adjoint_workspace(const tsu_grid* g, int dtype, int form, int64_t nsteps, int64_t ckpt_every, int32_t nrec,
                          size_t* bytes);

/* Reverse-time discrete adjoint of the forward run "tsu_init(u0, u1) then tsu_step_n(nsteps-1)"
 * for a receiver functional J(traces) (the paper has no adjoint; it is the exact reverse of the
 * scheme above, with multipliers lam^n = g^n + (2I + B) lam^{n+1} - lam^{n+2}; FP32 fields run the
 * same recursion in increment form, mu^n = lam^n - lam^{n+1} = mu^{n+1} + B lam^{n+1} + g^n).
 *   form      the form of that forward run (its checkpoints hold that form's two fields)
 *   nsteps    S (final state u^S); ckpt_every, ckpt: the checkpoint store the forward filled
 *             (tsu_ckpt_slots(S, every) slots); segments are recomputed from it
 *   u0        device [ny][ld], the forward's initial displacement (boundary read as 0)
 *   dtraces   device [S][nrec] of dtype: dJ/d(u^n at receiver r), n = 1..S
 *   g_hx, g_hy  device double [ny][ld], overwritten with dJ/dhx, dJ/dhy (FP64 accumulation;
 *             for FP32 fields FP32 partial sums over one segment are added into them)
 *   g_u0, g_u1  device [ny][ld] of dtype, overwritten with dJ/du0, dJ/du1
 * Every segment is recomputed from its checkpoint on a library-owned stream (one per device and
 * host thread, created by that thread's first call and destroyed when the thread exits)
 * concurrently with the reverse sweep of the previous one; all of it is ordered before the
 * call's last work on the caller's stream.
 * Errors: TSU_EINVAL, TSU_ENONPOS, TSU_ECFL, TSU_ENOMEM, TSU_ECUDA. */
int tsu_adjoint(const tsu_grid* g, int dtype, int form, double tau, const tsu_medium* m, int64_t nsteps,
                int64_t ckpt_every, const void* ckpt, const void* u0, int32_t nrec, const int64_t* rec_idx,
                const void* dtraces, double* g_hx, double* g_hy, void* g_u0, void* g_u1, void* ws, size_t ws_bytes,
                void* stream);

/* Diagnostic (the paper has no counterpart): the number of auxiliary streams the library holds
 * right now.  tsu_adjoint creates one per device and calling host thread, with five events, on
 * that thread's first call; they are destroyed when the thread exits. */
int tsu_aux_streams(void);

/* One problem of a batched family (all FP32, same form): grid, time step, medium, state (nbuf = 4,
 * initialised by tsu_init) and the number of steps to advance it. */
typedef struct {
  tsu_grid grid;
  double tau;
  tsu_medium medium;
  tsu_state* state;
  int64_t nsteps;
} tsu_problem;

/* Options of tsu_batch_run (NULL = defaults).  How the tiles of the family are packed into each
 * launch (order, rows) changes no result: every tile computes the same values wherever it runs. */
typedef struct {
  int32_t tdepth; /* steps per batched pass (0 = the kernel's default: 4 for kernel 2, 8 for kernel 3) */
  int32_t rows;   /* rows per chunk (0 = 80, halved down to 16 while the tiles do not fill the GPU) */
  int32_t kernel; /* 0 or 2: warp-blocked (tdepth 2 or 4); 3: CTA-blocked (tdepth 4 or 8) */
  int32_t graph;  /* 1: capture every launch of the call into one CUDA graph and launch that (needs a
                     non-default stream); 0: launch on the stream directly */
  int32_t order;  /* order of the tile table within problems of equal step counts:
                     0 problem by problem (each problem's chunks in turn, strips within a chunk),
                     1 every problem's full chunks first, the ragged last chunks at the end,
                     2 the problems interleaved chunk by chunk (chunk 0 of every problem, then 1 ...) */
  const int32_t* rows_per_problem; /* host [nprob] rows per chunk of each problem (>= 16; 0 = rows),
                                      or NULL for rows throughout */
} tsu_batch_opts;

/* Bytes of device workspace tsu_batch_run needs for these problems (descriptors and tile table). */
int tsu_batch_workspace(int32_t nprob, const tsu_problem* probs, const tsu_batch_opts* opts, size_t* bytes);

/* Advance a whole family of regularised problems (the eps-family (u_eps)_eps of Sec. 3.2, with
 * different singularities, widths, grid sizes and time steps) together: every launch of the
 * temporally blocked pass covers the tiles of all problems that still have tdepth steps to go;
 * leftover steps (nsteps % tdepth) run one per pass.  Each problem ends in the same state, bit for
 * bit, as tsu_step_n would leave it.  The call uploads descriptors (it synchronises with the
 * host once) and updates every state's cur/aux/step; tsu_sync_status(ws) reports expired waits.
 * Errors: TSU_EINVAL (mixed forms, non-FP32 fields, nbuf != 4), TSU_ENONPOS, TSU_ECFL, TSU_ENOMEM,
 * TSU_ECUDA. */
int tsu_batch_run(int32_t nprob, const tsu_problem* probs, const tsu_batch_opts* opts, void* ws, size_t ws_bytes,
                  void* stream);

/* tsu_step_n without a workspace, for callers that cannot allocate device memory (a host
 * application that owns the allocator and hands over only its buffers, a real-time loop that
 * must not stall on an allocation, a plugin whose host forbids it).  The paper has no
 * counterpart: this is an interface variant only.  It makes nsteps one-step passes exactly as
 * tsu_step_n does with kernel = 1 and opts->energy = energy (NULL: no energy), and takes the
 * energy-reduction scratch from a fixed array inside the library (256 B + 65536 FP64 partial
 * sums, kept on every device that uses the library until it is unloaded) instead of a workspace.
 *   - Grids needing more than 65536 partial sums (ceil(ld/512) * ceil((ny-2)/32) in FP32,
 *     ceil(ld/256) * ceil((ny-2)/32) in FP64) are refused with TSU_ENOMEM when energy is set.
 *   - The first call on a device looks up the array's device address with that device current;
 *     make that first call before any stream capture.
 *   - All calls on a device share the array and leave their last contents in it; each call zeroes
 *     what must start at zero.  Calls that overlap on the GPU race: order them.
 * It allocates nothing (no cudaMalloc, no library allocator).  Errors as tsu_step_n; the message
 * is in tsu_noalloc_last_error(). */
int tsu_step_n_noalloc(const tsu_grid* g, int dtype, double tau, const tsu_medium* m, tsu_state* st,
                       int64_t nsteps, double* energy, void* stream);
const char* tsu_noalloc_last_error(void);

/* Synchronise the stream, then read and clear the device status word in the workspace of
 * tsu_step_n or of the implicit calls: TSU_OK, or TSU_ETIMEOUT if a bounded device-side wait of a
 * kernel expired (that kernel stopped early; its outputs are invalid). */
int tsu_sync_status(void* ws, size_t ws_bytes, void* stream);

/* Energy E^{n-1/2} of the current pair (u^{n-1}, u^n) into energy_dev[0] (device double, or NULL)
 * and u^n at the receivers into trace (device [nrec], or NULL).  Does not step. */
int tsu_observe(const tsu_grid* g, int dtype, double tau, const tsu_medium* m, const tsu_state* st,
                double* energy_dev, int32_t nrec, const int64_t* rec_idx, void* trace, void* ws,
                size_t ws_bytes, void* stream);

/* ---- Implicit comparator (Sec. 3.3) -------------------------------------------------------
 * The paper solves its 2D problem with an implicit finite-difference scheme whose systems are
 * tridiagonal along grid lines (cyclic reduction), without writing the scheme out.  Read here as
 * the factorized scheme with weight sigma, in increment form:
 *   (I - sigma B_x)(I - sigma B_y) w^n = B u^n,   v^{n+1} = v^n + w^n,   u^{n+1} = u^n + v^{n+1},
 *   start: the same systems with B u^0, then v^1 = tau u1 + w^0 / 2, u^1 = u^0 + v^1,
 * where B_x u = tau^2/dx^2 fx(u) and B_y u = tau^2/dy^2 fy(u) are the two halves of B = tau^2 L_h
 * of the explicit scheme.  sigma >= 1/4 is stable for every tau (no Courant bound); sigma = 0 is
 * the explicit leapfrog.  Each factor is one tridiagonal system per grid line over the interior
 * nodes (zero Dirichlet ends).
 *
 * tsu_implicit_sizes: bytes of the factor buffer and of the workspace for this grid and dtype.
 *   Transposed fields have nx rows of ldT = roundup(ny, 32) elements; the factor holds
 *   [ny][ld] + 2 [nx][ldT] elements, the workspace a 256-byte header (its int at byte 4 is a
 *   status word) and [nx][ldT] + max(ny ld, nx ldT) elements.
 * tsu_implicit_factor: the line systems' pivots for (tau, sigma, medium), computed once on the
 *   device into `factor` (caller-owned, 16-byte aligned, factor_bytes >= the size above).  Any
 *   change of tau, sigma or the depth needs a new factor.
 * tsu_implicit_init: u0 (device [ny][ld]; boundary nodes ignored) and u1 (device or NULL = 0) ->
 *   buf[0] = u^1, buf[1] = v^1 (st->form must be TSU_FORM_INCREMENT, nbuf >= 2; u0 may be
 *   buf[0]); sets cur = 0, aux = 1, step = 1.
 * tsu_implicit_step_n: nsteps steps in place on buf[cur] (u) and buf[aux] (v); step += nsteps.  On a
 *   stream that can be captured (not the legacy or per-thread default stream, not capturing) a call
 *   of 4 steps or more runs its launches (two per step) as one CUDA graph; the executable graph is
 *   kept per host thread and launched again while calls repeat the same arguments (same grid,
 *   buffers, tau, sigma and nsteps).  FP32 grids of at most 129 x 129 nodes (256 x 256, ld and
 *   ldT <= 256) run every step of the call, and the start of tsu_implicit_init, in one launch of a
 *   cluster of 8 (16) CTAs that holds the fields in shared memory; its hand-overs between CTAs are waited for with a bound (2 s), and
 *   a wait that runs out ends the launch early with TSU_ETIMEOUT in the status word.  The results
 *   are the same on every path.
 * Every call is asynchronous on `stream`; the workspace (16-byte aligned, >= the size above,
 * zero-filled by the caller before its first use) is scratch that must not be shared by calls in
 * flight at the same time; tsu_sync_status(ws, ws_bytes, stream) reads and clears its status word.
 * Errors: TSU_EINVAL (arguments, form, alignment), TSU_ENONPOS (the medium's extrema), TSU_ECFL (sigma < 1/4 and
 * tau^2 (hx_max/dx^2 + hy_max/dy^2) (1 - 4 sigma) > 1), TSU_ENOMEM (factor or workspace too
 * small), TSU_ECUDA. */
int tsu_implicit_sizes(const tsu_grid* g, int dtype, size_t* factor_bytes, size_t* ws_bytes);
int tsu_implicit_factor(const tsu_grid* g, int dtype, double tau, double sigma, const tsu_medium* m, void* factor,
                        size_t factor_bytes, void* stream);
int tsu_implicit_init(const tsu_grid* g, int dtype, double tau, double sigma, const tsu_medium* m, const void* factor,
                      const void* u0, const void* u1, tsu_state* st, void* ws, size_t ws_bytes, void* stream);
int tsu_implicit_step_n(const tsu_grid* g, int dtype, double tau, double sigma, const tsu_medium* m,
                        const void* factor, tsu_state* st, int64_t nsteps, void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TSU_H */
