/*
 * wilson_eo.h -- C ABI of libwilson_eo.so, the even-odd preconditioned Wilson
 * fermion matrix on one GB300 GPU (sm_103a).
 *
 * The operator (Kanamori, Nitadori, Matsufuru, arXiv:2303.08609):
 *
 *   D_W(x,y) = delta_{x,y} - kappa sum_mu [ (1 - gamma_mu) U_mu(x) delta_{x+mu,y}
 *                                        + (1 + gamma_mu) U_mu^dag(x-mu) delta_{x-mu,y} ]
 *                                                         (Sec. 2, Eq. 1 and its footnote)
 *   H_eo, H_oe : the hopping sum of Eq. 1 without -kappa, restricted to
 *                odd->even and even->odd sites, so D_eo = -kappa H_eo, D_oe = -kappa H_oe
 *   M_eo       = 1 - D_ee^-1 D_eo D_oo^-1 D_oe = 1 - kappa^2 H_eo H_oe
 *                (Sec. 2, Eq. 4; D_ee = D_oo = 1 for the Wilson matrix)
 *
 * Conventions fixed by this library where the paper leaves them open:
 *   - lattice: periodic in all four directions; every extent even and >= 2;
 *     dims[] = {Lx, Ly, Lz, Lt}; V = Lx Ly Lz Lt;
 *   - parity: a site (x,y,z,t) is even when x+y+z+t is even (Sec. 3.3);
 *     the V/2 sites of one parity are numbered by i = lex/2 with
 *     lex = ((t Lz + z) Ly + y) Lx + x (compaction in x, Sec. 3.3, Fig. 4);
 *   - gamma basis: Euclidean chiral, gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]
 *     for k = x,y,z and gamma_t = [[0, 1], [1, 0]]; gamma_5 = diag(1,1,-1,-1);
 *   - projector signs as in Eq. 1: (1 - gamma_mu) on the forward neighbour.
 *
 * Canonical external layouts (complex numbers interleaved re, im):
 *   gauge   U[mu][lex][a][b]         mu = 0..3 (x,y,z,t), 4*V links of 3x3,
 *                                    complex128 (gauge_is_f64 = 1) or complex64
 *   spinor  psi[rhs][spin][colour][i] one parity, i = 0..V/2-1 fastest
 *                                    (planar: each of the 12 spin-colour
 *                                    components is a contiguous array of V/2
 *                                    sites), complex128 for WEO_F64 handles and
 *                                    complex64 for WEO_F32 / WEO_F16 / WEO_BF16;
 *                                    wilson_eo_spinor_layout converts from and
 *                                    to the site-major psi[rhs][i][spin][colour]
 *   force   F[mu][lex][a][b]         like the gauge field, in the spinor dtype
 *
 * Pointers: every array argument may be device memory (cudaMalloc / torch) or
 * host memory. Host arrays are copied through buffers the handle owns, on
 * `stream`. Calls are asynchronous on `stream` (a cudaStream_t, NULL = the
 * legacy default stream) unless stated otherwise: with device or page-locked
 * (pinned) host arrays the caller synchronises the stream before reading an
 * output; a pageable host output is complete when the call returns, and a
 * pageable host input may be reused as soon as the call returns.
 *
 * Ownership: the caller owns every array it passes. The handle owns its packed
 * gauge copies, its intermediate odd-site fields, solver workspaces, staging
 * buffers and tuning state, and frees them in wilson_eo_destroy. A handle may be
 * used from one host thread at a time, and its calls must be ordered on the
 * device (one stream, or streams synchronised by the caller), because calls
 * share the handle's intermediate buffers.
 *
 * Errors: every int-returning call returns WEO_OK (0) or a negative weo_status.
 * No call aborts, exits, throws across the ABI or traps on the device.
 * wilson_eo_last_error() describes the most recent failure of the calling thread.
 */
#ifndef WILSON_EO_H
#define WILSON_EO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wilson_eo_s *wilson_eo_t;

typedef enum {
    WEO_OK = 0,
    WEO_ERR_ARG = -1,           /* null pointer, nrhs < 1, bad enum, bad tolerance ... */
    WEO_ERR_DIMS = -2,          /* an extent odd or < 2, or a volume too large */
    WEO_ERR_UNSUPPORTED = -3,   /* combination not provided (e.g. batch of mixed precisions) */
    WEO_ERR_CUDA = -4,          /* a CUDA runtime call or kernel launch failed */
    WEO_ERR_NOT_CONVERGED = -5, /* solver hit maxiter; outputs hold the best iterate */
    WEO_ERR_NONFINITE = -6,     /* NaN or Inf met in a solver reduction */
    WEO_ERR_TIMEOUT = -7,       /* a bounded device-side wait gave up */
    WEO_ERR_OOM = -8            /* device or host allocation failed */
} weo_status;

/* Storage precision of the Dirac operator inside a handle. WEO_F16 / WEO_BF16
 * store spinors as 16-bit values scaled by a per-site FP32 norm (the maximum
 * modulus of the site's 24 reals) and links as plain 16-bit values; all
 * arithmetic is FP32. */
typedef enum { WEO_F64 = 0, WEO_F32 = 1, WEO_F16 = 2, WEO_BF16 = 3 } weo_prec;

/* Link storage: all 18 reals, or rows 0 and 1 only (12 reals) with row 2 rebuilt
 * in registers as conj(row0 x row1), exact for SU(3) up to rounding. */
typedef enum { WEO_LINK18 = 0, WEO_LINK12 = 1 } weo_linkfmt;

/* Create a handle for one lattice.
 *   out      receives the handle (set to NULL on failure)
 *   dims     {Lx, Ly, Lz, Lt}, each even and >= 2 (WEO_ERR_DIMS otherwise);
 *            V/2 must stay below 2^31
 *   kappa    hopping parameter of Eq. 1 (kappa = 1/(8 + 2m))
 *   prec     weo_prec; linkfmt weo_linkfmt
 *   gauge    canonical gauge field (4*V*9 complex), copied and packed; the caller
 *            may free it when the call returns
 * Blocks until the packed copy is complete. */
int wilson_eo_create(wilson_eo_t *out, const int dims[4], double kappa, int prec, int linkfmt,
                     const void *gauge, int gauge_is_f64, void *stream);

/* Replace the gauge field (same layout and rules as in create). */
int wilson_eo_set_gauge(wilson_eo_t h, const void *gauge, int gauge_is_f64, void *stream);

/* Change kappa (host-side state only; takes effect for later calls). */
int wilson_eo_set_kappa(wilson_eo_t h, double kappa);

/* Query: dims (int[4]), V/2, precision, link format, kappa, and the bytes the
 * handle holds on the device. Any output pointer may be NULL. */
int wilson_eo_info(wilson_eo_t h, int dims_out[4], long long *half_volume, int *prec,
                   int *linkfmt, double *kappa, size_t *device_bytes);

/* out_e = M_eo in_e = in_e - kappa^2 H_eo H_oe in_e   (Eq. 4)
 * in_e, out_e: nrhs canonical even spinors. out_e must not alias in_e.
 * nrhs >= 1; right-hand sides share the links, which are read once per site
 * for a block of right-hand sides. */
int wilson_eo_apply(wilson_eo_t h, void *out_e, const void *in_e, int nrhs, void *stream);

/* out_e = M_eo^dag in_e = gamma_5 M_eo gamma_5 in_e, the adjoint of Eq. 4
 * (gamma_5-hermiticity of Eq. 1). Same arguments and rules as apply. */
int wilson_eo_apply_dag(wilson_eo_t h, void *out_e, const void *in_e, int nrhs, void *stream);

/* One hopping term of Eq. 1 (no kappa): out = H_{po,1-po} in, onto the sites of
 * parity out_parity (0: H_eo, odd -> even; 1: H_oe, even -> odd), dag != 0 for
 * its adjoint. in and out are canonical single-parity spinors. Not provided for
 * 16-bit handles (WEO_ERR_UNSUPPORTED): their intermediates are internal. */
int wilson_eo_hop(wilson_eo_t h, int out_parity, int dag, void *out, const void *in, int nrhs,
                  void *stream);

/* Euclidean gradient of the real function L = Re<g_e, M_eo phi_e> with respect
 * to every link: grad[mu][lex][a][b] = dL/dRe U_mu(x)_ab + i dL/dIm U_mu(x)_ab
 * (the convention torch uses for real losses of complex tensors), obtained by
 * differentiating both hopping terms of Eq. 1 in M_eo = 1 - kappa^2 H_eo H_oe
 * (Eq. 4). grad: canonical gauge layout in the spinor dtype (4*V*9 complex).
 * With g_e = dLoss/d(M_eo phi_e) this is the link part of the backward pass.
 * FP64 and FP32 handles only (WEO_ERR_UNSUPPORTED otherwise). */
int wilson_eo_link_grad(wilson_eo_t h, void *grad, const void *g_e, const void *phi_e,
                        void *stream);

/* Pseudofermion force of S(U, phi) = |M_eo phi_e|^2 (the Schur-decomposed
 * determinant of Sec. 2 evaluated with a noise vector phi): force[mu][lex] is
 * the traceless anti-Hermitian 3x3 matrix F with dS/d eps = Re tr(X^dag F) for
 * every traceless anti-Hermitian X under U_mu(x) -> exp(eps X) U_mu(x), i.e.
 * F = TA(G U^dag) with G the link gradient for g_e = 2 M_eo phi_e and
 * TA(W) = (W - W^dag)/2 - tr(W - W^dag)/6. If dS_dphi_e is not NULL it receives
 * 2 M_eo^dag M_eo phi_e. Layouts as in wilson_eo_link_grad. FP64 / FP32 only. */
int wilson_eo_force(wilson_eo_t h, void *force, void *dS_dphi_e, const void *phi_e,
                    void *stream);

/* Solve M_eo^dag M_eo x_e = b_e (CG on the normal equations of the even
 * system of Eq. 4; Sec. 2 notes the solver's cost is that of the matrix
 * multiplication). x_e and b_e are canonical even spinors in complex128
 * whatever the handle's precision; x_e holds the initial guess on entry and the
 * solution on return.
 *   mixed = 0: plain FP64 CG (FP64 operator, vectors and reductions).
 *   mixed = 1: CG with the handle's low-precision operator (FP32 for FP64 and
 *              FP32 handles, FP16/BF16 storage for 16-bit handles) and FP32
 *              vectors, with reliable updates: whenever the iterated residual
 *              has fallen by `delta` (default 0.1) the FP32 increment is added
 *              to the FP64 solution and the residual is recomputed as b - A x
 *              with the FP64 operator. Reductions accumulate in FP64.
 * Convergence: |b - A x| / |b| <= tol with the residual recomputed in FP64 from
 * the returned x (true_relres_out). Returns WEO_OK, WEO_ERR_NOT_CONVERGED
 * (maxiter iterations done, or -- mixed mode -- the true residual grew 10^4-fold
 * above its best value because the low-precision operator is too far from the
 * FP64 one; x_e holds the last iterate), WEO_ERR_NONFINITE (NaN
 * or Inf, or a non-positive <p, A p>; x_e is not written) or an argument / CUDA
 * error. tol in (0, 1); maxiter >= 0. Blocks until done; the iterations run on
 * a stream the handle owns after the work already queued on `stream` finished.
 * Iterations are launched in chunks from a CUDA graph (see
 * wilson_eo_solver_config); the host reads one scalar per chunk. */
int wilson_eo_solve(wilson_eo_t h, void *x_e, const void *b_e, double tol, int maxiter, int mixed,
                    int *iters_out, double *true_relres_out, void *stream);

/* The full Wilson system D_W xi = eta (Eq. 2) through the even-odd route:
 *   wilson_eo_prepare_source: rhs_e = eta_e - D_eo eta_o = eta_e + kappa H_eo eta_o
 *                             (right-hand side of Eq. 4; D_ee = 1)
 *   wilson_eo_reconstruct:    xi_o  = eta_o - D_oe xi_e  = eta_o + kappa H_oe xi_e
 *                             (Eq. 5; D_oo = 1)
 * Both take canonical single-parity spinors in the handle's spinor dtype
 * (FP64 and FP32 handles; WEO_ERR_UNSUPPORTED for 16-bit) and are
 * asynchronous for device arrays. */
int wilson_eo_prepare_source(wilson_eo_t h, void *rhs_e, const void *eta_e, const void *eta_o,
                             void *stream);
int wilson_eo_reconstruct(wilson_eo_t h, void *xi_o, const void *eta_o, const void *xi_e,
                          void *stream);

/* Solve D_W xi = eta: prepare the even source with FP64 operators, solve
 * M_eo^dag M_eo xi_e = M_eo^dag rhs_e with wilson_eo_solve (same `mixed`, tol,
 * maxiter and status rules; xi_e holds the initial guess on entry), then
 * reconstruct xi_o in FP64. All four arrays are complex128 canonical spinors
 * (device or host). iters_out / relres_out describe the even solve (the odd
 * equations hold exactly up to rounding). Blocks until done; allocates three
 * temporary FP64 fields for the call. */
int wilson_eo_solve_full(wilson_eo_t h, void *xi_e, void *xi_o, const void *eta_e,
                         const void *eta_o, double tol, int maxiter, int mixed, int *iters_out,
                         double *relres_out, void *stream);

/* wilson_eo_solve for nrhs (1..64) right-hand sides at once: x_e and b_e hold
 * nrhs canonical complex128 even spinors. The systems run as independent CGs
 * in lockstep -- every operator application covers all of them, so the
 * multi-right-hand-side hop kernels read each link once for a block of
 * right-hand sides -- each with its own scalars, convergence and restarts.
 * iters_out[r] and true_relres_out[r] (arrays of nrhs, may be NULL) give the
 * iteration at which system r met tol and its FP64 true residual. Status as in
 * wilson_eo_solve; WEO_ERR_NOT_CONVERGED if any system missed tol. */
int wilson_eo_solve_multi(wilson_eo_t h, void *x_e, const void *b_e, int nrhs, double tol,
                          int maxiter, int mixed, int *iters_out, double *true_relres_out,
                          void *stream);

/* Solver settings: reliable-update threshold delta in (0, 1), iterations per
 * chunk (>= 1; default 8), use_graphs 1/0 (default 1). A value outside its range
 * leaves that setting unchanged. */
int wilson_eo_solver_config(wilson_eo_t h, double delta, int chunk, int use_graphs);

/* How the mixed-precision solver forms the true residual b - A x of a
 * reliable update: mode 1 (default) with the float-float operator of
 * wilson_eo_apply_ff64 (FP64-class accuracy, several times faster than native
 * FP64 on GPUs with a reduced FP64 rate), and whenever that residual says a
 * system has met tol, once more with the native FP64 operator, which alone
 * decides convergence; mode 0 with the native FP64 operator every time. Plain
 * FP64 solves always use the native FP64 operator. Other modes: WEO_ERR_ARG. */
int wilson_eo_solver_residual(wilson_eo_t h, int mode);

/* Search direction of the mixed-precision solver after a reliable update:
 * restart 0 keeps it (Clark et al. 2010); restart 1 starts a new direction from
 * the recomputed residual at every reliable update, which makes the solve a
 * defect correction whose inner solves reduce the residual by `delta` each;
 * restart 2 (default) restarts for BF16 inner operators and keeps the direction
 * otherwise. Measured at 48^3 x 96, kappa = 0.135: with BF16 links (unit
 * roundoff 2^-8) kept directions make the iteration diverge from the FP64
 * system, restarted ones converge in 264 iterations; FP16 converges either way
 * and is faster keeping them (224 iterations). Sec. 2 leaves the solver open.
 * Other values: WEO_ERR_ARG. */
int wilson_eo_solver_restart(wilson_eo_t h, int restart);

/* Statistics of the handle's last solve: low-precision (or FP64 in plain mode)
 * CG iterations, reliable updates, native FP64 operator applications (true
 * residuals), float-float operator applications (true residuals of reliable
 * updates, see wilson_eo_solver_residual), wall seconds. Any pointer may be
 * NULL. */
int wilson_eo_solve_stats(wilson_eo_t h, int *iterations, int *reliable_updates,
                          int *fp64_applies, int *ff_applies, double *seconds);

/* M_eo (dag = 0) or M_eo^dag on n lattices at once, in ONE persistent
 * cooperative kernel launch: every lattice keeps its own extents, kappa and
 * links (its handle); the launch covers all first hops (Eq. 1 onto odd sites),
 * synchronises the grid, then all second hops with the diagonal term (Eq. 4).
 *   n        1..24 handles, all FP64 or all FP32, one link format, created on
 *            the current device, no handle twice
 *   outs[k], ins[k]  device arrays: one canonical even spinor of lattice k
 * Uses each handle's odd-site buffer. Asynchronous on `stream`. */
int wilson_eo_apply_batch(int n, const wilson_eo_t *hs, void *const *outs,
                          const void *const *ins, int dag, void *stream);

/* wilson_eo_apply_batch with nrhs[k] (1..1024) right-hand sides for lattice k
 * (outs[k], ins[k] hold nrhs[k] canonical even spinors), still one cooperative
 * launch; for FP32 handles two right-hand sides share each link load. */
int wilson_eo_apply_batch_rhs(int n, const wilson_eo_t *hs, void *const *outs,
                              const void *const *ins, const int *nrhs, int dag, void *stream);

/* Autotune M_eo on this handle with nrhs right-hand sides: every candidate is
 * timed with CUDA events on `stream` and the fastest is kept -- the two-launch
 * algorithm with threads 64/128/192/256 per CTA and 1, 2 or 4 right-hand sides
 * per thread or 2 on neighbouring lanes (FP32 / 16-bit handles, nrhs >= 2), and
 * for FP32 / 16-bit handles the fused algorithm with a lookahead of 4 or 8
 * t-slices and 128 / 256 threads, and for FP32 18-real handles with nrhs = 1
 * the TMA-staged hop (wilson_eo_get_launch, wilson_eo_get_algorithm,
 * wilson_eo_get_staging). threads_out / rhs_block_out describe the winner. Results
 * are cached per process by (GPU, extents, precision, link format, nrhs) and,
 * if the environment variable WILSON_EO_TUNE_CACHE names a file, appended to it
 * and read back by later processes. Allocates two temporary spinor fields.
 * Any output pointer may be NULL. Blocks until done. */
int wilson_eo_tune(wilson_eo_t h, int nrhs, int *threads_out, int *rhs_block_out, double *ms_out,
                   void *stream);

/* Choose how M_eo and M_eo^dag are computed for FP32, FP16 and BF16 handles
 * (apply, apply_dag, force, and the inner operator of the mixed solver):
 *   algo 0  two hop launches with the odd-site intermediate in HBM (default);
 *   algo 1  one persistent launch for both hops of Eq. 4: CTAs take (hop,
 *           t-slice, chunk) items from a queue in which the first hop H_oe
 *           runs `lookahead` t-slices ahead of the second (1..64, clamped to
 *           Lt-1; 0 keeps the current value, default 4), so the second hop
 *           finds the links and the odd-site intermediate of its slices still
 *           in L2; `threads` per CTA 128 or 256 (0 keeps the current value).
 *           Same arithmetic and intermediate format as algo 0, so the
 *           results are bitwise equal.
 *   algo 2  the same wavefront of both hops in one persistent launch fed by
 *           the tensor-memory accelerator (FP32 handles with 18-real links and
 *           lattices the staged hop tiles, see wilson_eo_set_staging): per tile
 *           item one producer thread copies the neighbour spinor rows (tensor
 *           boxes) and the tile's links into a ring of shared-memory stages,
 *           and second-hop items wait until the first-hop items of slices
 *           t-1, t, t+1 have published. The links of both hops come from one
 *           pair block per tile (each link stored once, plus the row below
 *           each tile: 576 T + 144 Lx/2 bytes per tile of T sites), so a link
 *           leaves HBM once per M_eo. The blocks are built on first use (not
 *           while the stream is being captured) and after set_gauge.
 *           `lookahead` as for algo 1; `threads` is ignored.
 * Items wait for the items they depend on with bounded polling; if a wait ever
 * gives up (about a second without progress), the kernel records an error
 * that wilson_eo_check reports as WEO_ERR_TIMEOUT. FP64 handles: algo 1 gives
 * WEO_ERR_UNSUPPORTED; algo 2 gives it for any handle it cannot serve. */
int wilson_eo_set_algorithm(wilson_eo_t h, int algo, int lookahead, int threads);

/* Failure-path test of the fused kernel: runs one fused M_eo in which the
 * first-hop items never publish their completion (a flag that nothing sets) and
 * the poll limit is short (~0.3 ms), so the second-hop items' bounded waits run
 * out; the kernel records the error and every CTA returns. wilson_eo_check then
 * reports WEO_ERR_TIMEOUT. out_e receives garbage. Nothing faults, traps or
 * hangs; the context stays usable. FP32 / 16-bit handles, device arrays. With
 * algo 2 selected (wilson_eo_set_algorithm) the same test runs the fused
 * staged launch: its first-hop tiles never publish, the producers' bounded
 * waits for them give up after ~2 ms, every consumer group is stopped and the
 * CTAs return. */
int wilson_eo_inject_fused_timeout(wilson_eo_t h, void *out_e, const void *in_e, void *stream);

/* Hopping kernel fed by TMA (Eq. 1 for one parity, as wilson_eo_hop; used by
 * every hop of M_eo, M_eo^dag, the solvers and the force whose spinors are FP32
 * with 18-real FP32 links and one right-hand side). staged = 1: the output
 * sites are cut into tiles of R lattice rows; one producer thread per CTA
 * loads each tile's neighbour-spinor rows (same plane, y-1 / y+R rows, planes
 * z+-1 and t+-1) and the axpy addend as cp.async.bulk.tensor boxes, and the
 * tile's eight links per site as one cp.async.bulk copy of a link block, into
 * a ring of shared-memory stages; consumer warps compute from shared memory.
 * The link blocks are repacked from the handle's field when staging is turned
 * on and after wilson_eo_set_gauge (2 x 576 bytes per output site: 1.2 GB at
 * 32^3 x 64; each link is stored for both sites it joins; released by
 * staged = 0 and wilson_eo_destroy). Same arithmetic per direction as the default kernel; the
 * x/y and z/t halves of the sum are added at the end, so results agree to
 * FP32 rounding, not bitwise. Needs Lx/2 even and some R >= 2 dividing Ly with
 * R * Lx/2 <= 64 (WEO_ERR_UNSUPPORTED otherwise); arrays whose addresses are
 * not 16-byte aligned fall back to the default kernel. Waits are bounded
 * (about a second); a wait that gives up is reported by wilson_eo_check as
 * WEO_ERR_TIMEOUT. staged = 0 (default) restores the default kernel.
 * staged = 2 also stages multi-RHS hops: each tile's link block is loaded once
 * into one of two link slots and serves every right-hand side, whose spinor
 * boxes pass through a ring of 2-3 stages (measured slower than two right-hand
 * sides per thread at 12 right-hand sides on 32^3 x 64, 11.6 vs 13.7 TFlop/s,
 * so staged = 1 leaves multi-RHS hops to the default kernels).
 * rows: lattice rows R per tile (0: the largest that qualifies); depth: stages
 * of the ring, 2..5 (0: the most up to 3 that fit). A tile of R Lx/2 sites is
 * computed by one or two teams of two warps (x/y and z/t directions, 32 sites
 * each); each stage has its own teams, at most six per CTA, and all stages
 * must fit in 227 KB of shared memory (WEO_ERR_UNSUPPORTED otherwise). */
int wilson_eo_set_staging(wilson_eo_t h, int staged, int rows, int depth);

/* Whether staging is on, and the tile rows and ring depth the handle's lattice
 * resolves to (0, 0 when it cannot use the staged hop). Pointers may be NULL. */
int wilson_eo_get_staging(wilson_eo_t h, int *staged, int *rows, int *depth);

/* Failure-path test of the staged hop: one hop D_oe (in_e even, out_o odd,
 * device arrays, FP32 18-real handle on an eligible lattice) whose producer
 * never loads the first tile of each CTA and whose wait limit is 2 ms: the
 * consumers of that stage give up, the producer then gives up waiting for them
 * and waits for its own loads in flight, every CTA returns, and wilson_eo_check
 * reports WEO_ERR_TIMEOUT. out_o receives partial garbage. Nothing faults,
 * traps or hangs; the context stays usable. */
int wilson_eo_inject_staged_timeout(wilson_eo_t h, void *out_o, const void *in_e, void *stream);

/* Current algorithm (0 two launches, 1 fused), fused lookahead and threads. */
int wilson_eo_get_algorithm(wilson_eo_t h, int *algo, int *lookahead, int *threads);

/* Wait for `stream` and report whether any fused launch of this handle since
 * the previous check gave up a bounded wait (WEO_ERR_TIMEOUT: the outputs of
 * those calls are invalid); clears the record. WEO_OK otherwise. */
int wilson_eo_check(wilson_eo_t h, void *stream);

/* Current launch configuration of the handle's hopping kernels: threads per
 * CTA, right-hand sides per thread, right-hand sides on neighbouring lanes
 * (wilson_eo_set_launch, wilson_eo_set_rhs_lanes). Any pointer may be NULL. */
int wilson_eo_get_launch(wilson_eo_t h, int *threads, int *rhs_block, int *lanes);

/* The hopping term of wilson_eo_hop computed as on `ranks` sub-domains of the
 * lattice split along t (ranks divides Lt), with every t-hop that crosses a
 * sub-domain boundary -- the periodic wrap included, so ranks = 1 exchanges
 * with itself, as the forced communication of the paper's benchmark (Sec. 4)
 * -- passed through face buffers: pack (EO1: forward faces projected, backward
 * faces projected and multiplied by U^dag, Secs. 3.5-3.6), one device copy per
 * face and rank, bulk hops inside each sub-domain, and the boundary finish
 * (EO2). The result equals wilson_eo_hop up to rounding; it exercises the data
 * path a multi-GPU split would use. FP64 / FP32 handles, device arrays, one
 * right-hand side. */
int wilson_eo_hop_split(wilson_eo_t h, int ranks, int out_parity, int dag, void *out,
                        const void *in, void *stream);

/* Launch configuration of the hopping kernels for the handle's precision:
 * threads per block (32..256, a multiple of 32) and right-hand sides per
 * thread (1, 2 or 4; values other than 1 apply to FP32 and 16-bit handles, where the
 * links loaded for a site are shared by that many right-hand sides).
 * order 1 (default): the second hop of M_eo walks the sites from the top down,
 * so it first reads the part of the odd intermediate the first hop wrote last,
 * while that part is still in L2; order 0: both hops walk upward.
 * wilson_eo_tune sets threads and rhs_block from measurements. */
int wilson_eo_set_launch(wilson_eo_t h, int threads, int rhs_block, int order);

/* Right-hand sides on neighbouring lanes (FP32 and 16-bit handles): with
 * lanes = 2, 4 or 8, that many consecutive threads of a CTA take the same site
 * and different right-hand sides of a multi-RHS apply, so each link is fetched
 * once per warp for all of them while every thread keeps one right-hand side's
 * registers. Used when rhs_block is 1; clamped to nrhs. lanes = 1 (default)
 * turns it off. WEO_ERR_ARG for other values, WEO_ERR_UNSUPPORTED for lanes > 1
 * on an FP64 handle. */
int wilson_eo_set_rhs_lanes(wilson_eo_t h, int lanes);

/* Site order of the one-site-per-thread hopping kernels (every precision):
 * blocked 0 (default) gives each CTA consecutive parity indices, i.e. whole
 * rows of one (z, t) plane; blocked 1 gives each CTA of 8 Lx/2 threads the
 * rows (y0 + dy, z0 + dz, t0 + dt), dy, dz, dt in {0, 1}, so that half of its
 * y, z and t neighbour rows are rows it reads anyway and come from L1 rather
 * than L2 (Sec. 3.2 blocks sites in x and y for the same reason). Used when
 * 64 <= 8 Lx/2 <= 256; the CTA size then replaces wilson_eo_set_launch's
 * `threads`. The results do not depend on it. WEO_ERR_ARG for other values.
 * wilson_eo_tune times it too. */
int wilson_eo_set_site_blocks(wilson_eo_t h, int blocked);

/* Several right-hand sides with each tile's links loaded once (the batching
 * pattern of the multi-RHS hop; Table 1's tiling sweep is the paper's
 * analogue, Sec. 4): a CTA of 256 threads takes a tile of 256 / groups
 * consecutive output sites, copies the eight links of every tile site into
 * shared memory (as FP32, 576 bytes per site), and then passes over the tile,
 * its `groups` thread groups each taking rhs_per_thread right-hand sides per
 * pass (1, or 2 sharing every link read from shared memory; 2 is used when
 * nrhs >= 2 groups), until all nrhs are done; spinors are read from global
 * memory. groups 2, 4 or 8 turns it on for the handle's FP32 or 16-bit hops
 * whenever nrhs >= 2 (and sets one right-hand side per thread for the other
 * kernels); 0 (default) turns it off. WEO_ERR_ARG for other values,
 * WEO_ERR_UNSUPPORTED on an FP64 handle. wilson_eo_tune times these
 * configurations too. */
int wilson_eo_set_tile_links(wilson_eo_t h, int groups, int rhs_per_thread);
/* The handle's current groups (0 = off) and right-hand sides per thread. */
int wilson_eo_get_tile_links(wilson_eo_t h, int *groups, int *rhs_per_thread);

/* M_eo in_e (dag = 0) or M_eo^dag in_e (dag = 1) in float-float arithmetic:
 * every real is carried as an unevaluated sum hi + lo of two floats (about 48
 * significant bits; error-free two-sum and FMA-based two-product), so the
 * result has FP64-class accuracy (relative error ~1e-14) while all arithmetic
 * runs on the FP32 pipes. Works on any handle, whatever its precision: the
 * links come from the handle's canonical gauge field, split into float-float
 * once (4V x 144 bytes, kept until set_gauge). in_e / out_e: nrhs canonical
 * complex128 even spinors (host or device, as for wilson_eo_apply); the
 * handle keeps three float-float work fields of the same size. Same errors
 * as wilson_eo_apply. */
int wilson_eo_apply_ff64(wilson_eo_t h, void *out_e, const void *in_e, int nrhs, int dag, void *stream);

/* Per-kernel timing. With profiling on, every kernel the handle launches is
 * bracketed by two CUDA events on its stream (a few microseconds of host time
 * per launch). wilson_eo_profile_read waits for the recorded events and reports
 * up to max_kernels entries: kernel label (names + k*name_len, NUL-terminated),
 * summed device milliseconds and launch count; reset != 0 clears the totals. */
int wilson_eo_profile(wilson_eo_t h, int enable);
int wilson_eo_profile_read(wilson_eo_t h, int max_kernels, char *names, int name_len,
                           double *total_ms, long long *launches, int *n_kernels, int reset);

/* M_eo in_e (dag = 0) or M_eo^dag in_e (dag = 1) in FP32 without allocating
 * any memory. The paper has no counterpart: this entry point is for callers
 * that cannot call cudaMalloc -- code whose device memory belongs to a
 * framework's allocator, a real-time loop that must not enter the driver's
 * allocator, a plug-in that is only handed buffers. It takes no handle (creating
 * one allocates); the caller passes device arrays only:
 *   dims   {Lx, Ly, Lz, Lt}, each even and >= 2, and V/2 <= 349525 sites;
 *          larger lattices are rejected with WEO_ERR_DIMS and a message naming
 *          the limit
 *   gauge  canonical gauge field, complex64, device memory
 *   in_e   one canonical FP32 even spinor (planar complex64), device memory
 *   out_e  receives the result; must not alias in_e
 * All three arrays must be memory of the current device (or managed memory);
 * host arrays (staging them would allocate) and arrays of another GPU are
 * rejected with WEO_ERR_ARG before anything is launched.
 * The odd-site intermediate H_oe in_e lives in a fixed 32 MiB array compiled
 * into the library (a file-scope __device__ variable), which every GPU that
 * loads the library holds until the process exits. The first call on a device
 * looks up that array's device address for the current device and keeps it;
 * make that first call before any stream capture. The kept address dies with
 * the device's context: do not call this entry point on a device after
 * cudaDeviceReset of that device in the same process. All calls share the array and it keeps the
 * last call's contents; nothing in it has to start at zero because each call
 * writes every entry before reading it. Calls that overlap on the GPU (streams
 * without ordering between them, or several host threads) race on the array:
 * the caller must serialise them. Asynchronous on `stream`. */
int wilson_eo_apply_noalloc(const int dims[4], double kappa, const void *gauge, void *out_e,
                            const void *in_e, int dag, void *stream);

/* Reorder single-parity spinors between the site-major layout
 * psi[rhs][i][spin][colour] (each site's 12 spin-colour components together)
 * and this library's planar layout psi[rhs][spin][colour][i] (every call above
 * takes planar arrays), with the same parity index i = lex/2 (Sec. 3.3) in both.
 *   half_volume  V/2, the sites of one parity (>= 1)
 *   nrhs         right-hand sides (1..65535), stored one after the other
 *   elem_bytes   8 (complex64) or 16 (complex128)
 *   to_planar    1: src site-major -> dst planar; 0: src planar -> dst site-major
 *   dst, src     device arrays of half_volume * 12 * nrhs elements; must not overlap
 * Host arrays, overlapping arrays and values out of range: WEO_ERR_ARG, before
 * any launch. No counterpart in the paper (it fixes no in-memory order of the
 * components); a transpose through shared memory, asynchronous on `stream`,
 * allocates nothing. */
int wilson_eo_spinor_layout(long long half_volume, int nrhs, int elem_bytes, int to_planar,
                            void *dst, const void *src, void *stream);

/* Measured arithmetic peak of the current GPU in flop/s (2 per fused
 * multiply-add) for prec WEO_F64 or WEO_F32, written to *flops_per_s. A
 * measurement aid with no counterpart in the paper: the FP64 hopping kernels
 * are bound by the FP64 FMA rate rather than by memory on GPUs whose FP64 rate
 * is a small fraction of their FP32 rate, and their roofline is taken against
 * this number. Runs a short calibration launch, then ~100 ms of independent
 * FMA chains on every SM, on `stream`; synchronises with the stream before it
 * returns. Other precisions: WEO_ERR_ARG. */
int wilson_eo_alu_peak(int prec, double *flops_per_s, void *stream);

/* Measured read bandwidth from L2 into the SMs of the current GPU, in bytes/s:
 * every SM streams a 48 MiB buffer (resident in L2 after a warm-up pass) with
 * 16-byte L2-only loads, 40 passes, timed with CUDA events on `stream`. A
 * measurement aid with no counterpart in the paper: the hopping kernels re-read
 * neighbour spinors and links from L2 several times per site, and this is the
 * second roofline they are reported against. Allocates and frees its buffer;
 * synchronises with the stream before it returns. */
int wilson_eo_l2_peak(double *bytes_per_s, void *stream);

/* Release everything the handle owns (synchronises the device first).
 * NULL is accepted. */
void wilson_eo_destroy(wilson_eo_t h);

/* Static description of a weo_status value. */
const char *wilson_eo_strerror(int status);

/* Message of the most recent failure in the calling thread ("" if none). */
const char *wilson_eo_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* WILSON_EO_H */
