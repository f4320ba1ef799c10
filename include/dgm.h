/*
 * dgm.h -- C ABI of the GB300 library for the energy-conserving discontinuous
 * Galerkin (DG) discretisation of the time-domain Maxwell equations
 * (Koutschan, Lehrenfeld, Schoeberl, "Computer Algebra meets Finite Elements:
 * an Efficient Implementation for Maxwell's Equations", arXiv:1104.4208).
 *
 * Problem statement (Sec. 2, Sec. 3): a tetrahedral mesh, piecewise constant
 * permittivity eps and permeability mu per element, a polynomial order p and
 * initial fields go in; the fields after N explicit time steps and the
 * discrete energy come out.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - p is the polynomial degree of E; H has degree p-1 (Sec. 2: E in V^{k+1},
 *    H in V^k), or p with the equal_order option.  1 <= p <= DGM_PMAX.
 *  - Element map: the four vertices of each tetrahedron are re-ordered by
 *    ascending vertex key (vertex_key[v] if given, else the vertex id v);
 *    Phi(xh) = X0 + F xh, F = [X1-X0, X2-X0, X3-X0] (Sec. 3.2.1).
 *  - Fields are covariant (Sec. 3.2.1):  E|_T(x) = F^{-T} sum_a c_{m,a} e_m
 *    phi_a(Phi^{-1} x), phi_a the Dubiner basis of Sec. 4.2.2 exactly as
 *    printed (unnormalised), multi-indices a = (i,j,k), i+j+k <= p, ordered
 *    lexicographically with i outermost and k innermost.
 *  - Canonical field layout (host and device arrays, FP64):
 *      E [nt][3][N3(p)],  H [nt][3][N3(p-1)] (N3(p) with equal_order),
 *      N3(q) = (q+1)(q+2)(q+3)/6.
 *  - Face unknowns H^F (stabilized flux only): H^F = sum_g psi_g (K_1g t^1 +
 *    K_2g t^2) with psi the 2D Dubiner basis of Eq. (4) in the face
 *    parametrisation x = X_a + s t_1 + u t_2, t_1 = X_b - X_a, t_2 = X_c - X_a
 *    (a, b, c = the face's vertices by ascending key, coordinates taken from the
 *    first element that lists the face), t^i the dual basis of (t_1, t_2).
 *    Layout K [nfaces][2][N2(p)], N2(p) = (p+1)(p+2)/2; faces numbered by first
 *    occurrence when scanning elements in order and local faces 0..3 (local face
 *    f is opposite the f-th vertex in key order).
 *  - Faces without a partner are perfect electric conductor (PEC) walls.
 *
 * Errors: every function returns DGM_OK (0) or a negative DGM_ERR_* code and
 * leaves a message retrievable with dgm_last_error() (thread local).  No
 * exception crosses this boundary.
 *
 * Ownership: handles own their device memory.  Functions taking host arrays
 * copy them; functions named *_device take raw device pointers (e.g. from
 * torch tensors), never free them and are ordered on the given CUDA stream.
 * Handles are not thread safe.
 */
#ifndef DGM_H
#define DGM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DGM_PMAX 8

enum dgm_status {
    DGM_OK = 0,
    DGM_ERR_INVALID_ARG = -1,
    DGM_ERR_OOM = -2,
    DGM_ERR_CUDA = -3,
    DGM_ERR_UNSTABLE = -4,
    DGM_ERR_TIMEOUT = -5,
    DGM_ERR_UNSUPPORTED = -6
};

/* Numerical flux (Sec. 2.1): the central flux, or the stabilized central flux
 * with the additional face unknown H^F. */
enum dgm_flux { DGM_FLUX_CENTRAL = 0, DGM_FLUX_STABILIZED = 1 };

/* Arithmetic of the per-step operator.  FP64: state and arithmetic in double.
 * FP32: state and operator arithmetic in float; geometry, tables (rounded once)
 * and the energy reduction in double.
 * TC32: float state; the reference operators are applied to tiles of 128
 * elements on the tensor cores with TF32 operands (10-bit mantissa) and FP32
 * accumulation; one rounded table serves C_h and C_h^T, so the discrete
 * operator stays skew; geometry in double, per-element energy partials in float
 * summed in double.  Central flux, p <= 6.
 * TC16: as TC32, but the tensor-core operands are fp16 (also 10-bit mantissa,
 * range 6e-8 .. 65504): fp16 copies of E and H written next to the float
 * state, fp16 tables and face-trace buffers, fp16 MMAs with K = 16 and FP32
 * accumulation; the update and the energy use the float state.  The
 * orthonormalised coefficients and face traces must stay inside the fp16 range
 * (magnitudes well below 65504, and far above 6e-8 to keep their precision):
 * the equations are linear, so scale the fields into that range.  An overflow
 * shows as DGM_ERR_UNSTABLE from dgm_run when energies are requested.
 * By default (variant 0) TC16 runs the resident-table kernels: the operators
 * are split by field component -- the three reference derivatives of the
 * curl (Sec. 3.2.2) and one trace matrix per face (Sec. 3.2.3), signed by the
 * reference face tangents -- and the whole set stays in shared memory, one
 * CTA per SM.  Variant 1 selects the dense-operator kernels of TC32 with fp16
 * operands (the operators streamed through a copy ring per tile).
 * TCBF16: the resident-table kernels with bf16 operands (8-bit mantissa,
 * fp32's range: no scaling needed; operand rounding 8x coarser than fp16).
 * TC16X2: the dense-operator kernels with fp16 field operands and two-term
 * reference tables: every table value v is held as hi = fp16(v) plus
 * lo = fp16(v - hi) (about 22 significant bits), and every table MMA runs
 * twice, hi and lo, into the same FP32 accumulator.  The rounding of the
 * tables, which perturbs the operator itself and accumulates as a phase error
 * over long runs, drops by about three orders of magnitude; the fields'
 * operand rounding stays that of TC16.  About twice the table traffic of TC16.
 * Central flux, p <= 6 for every tensor-core precision. */
enum dgm_precision {
    DGM_PREC_FP64 = 0,
    DGM_PREC_FP32 = 1,
    DGM_PREC_TC32 = 2,
    DGM_PREC_TC16 = 3,
    DGM_PREC_TCBF16 = 4,
    DGM_PREC_TC16X2 = 5
};

typedef struct dgm_options {
    int flux;           /* dgm_flux */
    double alpha0;      /* alpha = alpha0 * p^2 (Sec. 2.1: alpha grows like p^2) */
    int precision;      /* dgm_precision */
    int variant;        /* 0 = automatic kernel choice (dgm_autotune may change it);
                           TC16: 1 = dense-operator kernels; FP64/FP32 with the central flux:
                           1 = dense curl, 2 = sparse curl (the exact zeros of D_x, D_y, D_z
                           skipped, Sec. 4.2.2), 3 = element-group kernels (sparse curl; a block
                           takes 32 elements at a time, lane e of each warp working on element
                           e, so every multiply-add has all 32 lanes busy; not with the
                           compensated update, DGM_ERR_UNSUPPORTED where a block's shared
                           memory cannot hold 32 elements at this degree) */
    int checks;         /* reserved: accepted, no effect.  Inputs are always validated at
                           creation; an unstable dt shows as DGM_ERR_UNSTABLE from the energy
                           watchdog of dgm_run (energies requested), and dgm_estimate_dt
                           gives the bound */
    int compensated;    /* FP32 with the central flux only (else DGM_ERR_UNSUPPORTED if set):
                           Kahan-compensated time-step update.  Every coefficient of E and H
                           carries a float compensation term holding the rounding error of its
                           last update, which is fed back into the next one, so the state
                           accumulates increments to about twice float precision; 8 extra
                           bytes of traffic per coefficient and step.  Default 0 */
    int equal_order;    /* FP64 and FP32 only (else DGM_ERR_UNSUPPORTED if set): H of degree p
                           like E (E, H in V^k x V^k) instead of p - 1 (Sec. 2: V^{k+1} x V^k).
                           The same scheme of Sec. 2.1 and Sec. 3 on the other pair of spaces:
                           N3(p) coefficients per component for both fields, face traces of
                           degree p on both sides.  Use it with the stabilized flux: with the
                           central flux this pair keeps spurious modes.  Default 0 */
} dgm_options;

typedef struct dgm_ctx dgm_ctx;
typedef struct dgm_mesh dgm_mesh;
typedef struct dgm_problem dgm_problem;

/* Library version (major*10000 + minor*100 + patch). */
int dgm_version(void);

/* Message of the last failing call on this thread ("" if none). */
const char* dgm_last_error(void);

/* Fill *opt with defaults: central flux, alpha0 = 1, FP64, automatic variant,
 * no compensation. */
void dgm_default_options(dgm_options* opt);

/* Context bound to CUDA device `device`.  DGM_ERR_CUDA if the device is absent. */
int dgm_create(dgm_ctx** ctx, int device);
int dgm_destroy(dgm_ctx* ctx);

/* Mesh (Sec. 2: triangulation T_h of tetrahedra, facets F_h).
 * xyz [nv][3] vertex coordinates; tets [nt][4] vertex ids; vertex_key [nv]
 * (nullable) identifies periodic copies of a vertex -- two faces whose three
 * keys coincide are glued (the periodic translation is implied by the
 * coordinates).  Faces without a partner are PEC walls.
 * The mesh is host data: ctx may be NULL (no GPU is touched).
 * Errors: DGM_ERR_INVALID_ARG for ids out of range, repeated keys in one tet,
 * degenerate tets (|det F| <= 1e-12 (max edge component)^3), faces shared by
 * more than two tets, a tet glued to itself. */
int dgm_mesh_create(dgm_ctx* ctx, int64_t nv, const double* xyz, int64_t nt,
                    const int32_t* tets, const int32_t* vertex_key, dgm_mesh** out);
int dgm_mesh_destroy(dgm_mesh* mesh);
/* Counts: elements, faces, boundary (PEC) faces.  Any pointer may be NULL. */
int dgm_mesh_info(const dgm_mesh* mesh, int64_t* nt, int64_t* nfaces, int64_t* nboundary);

/* Problem: mesh + p + eps[nt] + mu[nt] (> 0) + options (nullable: defaults).
 * Builds the reference tables for p (Sec. 3.2.2, Sec. 3.2.3), the per-element
 * inverse mass blocks (Sec. 3.3.1) and uploads everything to the device.
 * Fields start at zero. */
int dgm_problem_create(dgm_ctx* ctx, const dgm_mesh* mesh, int p, const double* eps,
                       const double* mu, const dgm_options* opt, dgm_problem** out);
int dgm_problem_destroy(dgm_problem* prob);
/* Lengths (in doubles) of the canonical E, H and H^F arrays. */
int dgm_problem_sizes(const dgm_problem* prob, int64_t* nE, int64_t* nH, int64_t* nHF);

/* Copy fields in/out (canonical layout, FP64 host arrays).  HF may be NULL
 * (ignored / zero) and must be NULL for the central flux. */
int dgm_set_fields(dgm_problem* prob, const double* E, const double* H, const double* HF);
int dgm_get_fields(dgm_problem* prob, double* E, double* H, double* HF);
/* Same with device pointers (FP64, canonical layout), ordered on `stream`. */
int dgm_set_fields_device(dgm_problem* prob, const double* E, const double* H,
                          const double* HF, void* stream);
int dgm_get_fields_device(dgm_problem* prob, double* E, double* H, double* HF, void* stream);

/* One half of the symplectic Euler step of Sec. 3, applied in place:
 *   which = 0 (H-kick):  H += dt M_mu^{-1} C_h E   (and H^F += dt M_F^{-1} S E)
 *   which = 1 (E-kick):  E -= dt M_eps^{-1} C_h^T H (including the H^F term)
 * C_h is the DG curl with the chosen flux (Sec. 2.1).  Ordered on `stream`
 * (NULL = the legacy default stream). */
int dgm_kick(dgm_problem* prob, int which, double dt, void* stream);

/* nsteps leapfrog steps (symplectic Euler with H staggered by dt/2, Sec. 3),
 * started and finished with half kicks so that E, H are reported at the same
 * time t + nsteps*dt.  energy_out (nullable, host, nsteps+1 doubles) receives
 * the modified discrete energy
 *   W^n = 1/2 (eps E^n, E^n) + 1/2 (mu H^{n-1/2}, H^{n+1/2})
 *         [+ 1/2 sum_F (h_F/alpha) (H^{F,n-1/2}, H^{F,n+1/2})_F]
 * which the scheme conserves exactly up to round-off (Sec. 2.1, Eq. (2)).
 * Blocks until the energies are on the host when energy_out != NULL.  With
 * energies requested, a blow-up is reported as DGM_ERR_UNSTABLE: a recorded
 * energy that is not finite, or (no point source set) one above 10 W^0. */
int dgm_run(dgm_problem* prob, double dt, int64_t nsteps, void* stream, double* energy_out);

/* Higher-order symplectic time stepping (Sec. 3 leaves the explicit integrator
 * open; the spatial operator conserves energy, so symplectic compositions keep
 * the energy bounded).  order = 2: the leapfrog of dgm_run.  order = 4: every
 * step of size dt is the symmetric composition of three leapfrog steps of
 * sizes w1 dt, w0 dt, w1 dt with w1 = 1/(2 - 2^{1/3}), w0 = 1 - 2 w1 (the
 * triple-jump construction of Yoshida, 1990), with adjacent half kicks merged:
 * 3 E-kicks and 3 H-kicks per step.  The fields start and end synchronized, as
 * in dgm_run.  The substep |w0| dt = 1.70 dt must itself be stable, so dt is
 * bounded by about 0.59 of the leapfrog bound.  Point sources are not
 * supported (DGM_ERR_UNSUPPORTED): they are sampled at leapfrog midpoints.
 * Blocks until the steps are done; no energies are recorded (use dgm_energy). */
int dgm_run_composed(dgm_problem* prob, double dt, int64_t nsteps, int order, void* stream);

/* Stability bound of the explicit scheme (Sec. 3): dt <= 2 / sqrt(rho) with rho
 * the spectral radius of M_mu^{-1} C_h M_eps^{-1} C_h^T (face unknowns included
 * for the stabilized flux), estimated by `iters` power iterations (Sec. 3
 * leaves the estimate to an iterative eigenvalue method) that apply the
 * library's own E- and H-kicks.  The printed bound 2 rho^{-1} is read as
 * 2 rho^{-1/2} (dimensionally a time).  The state is saved and restored; the
 * start vector is a fixed pseudo-random H.  Blocks; allocates temporaries. */
int dgm_estimate_dt(dgm_problem* prob, int iters, double* rho, double* dt_max);

/* Resonance frequencies of the cavity: the frequency-domain problem of Sec. 2.2
 * (i omega eps E = curl H, i omega mu H = -curl E, PEC walls) discretised by the
 * DG operator of Sec. 2.1.  Eliminating H (and, for the stabilized flux, H^F)
 * gives omega^2 M_eps e = K e with K = C_H^T M_mu^{-1} C_H (+ S^T M_F^{-1} S),
 * symmetric positive semi-definite by the skew-adjointness of the scheme.
 * The smallest omega are found by `m` Lanczos steps on A = M_eps^{-1} K in the
 * M_eps inner product, with full reorthogonalisation (Gram-Schmidt twice per
 * step); each step applies A by one H-kick and one E-kick of the library's own
 * kernels with dt = 1 from E = v, H = 0.  Ritz values at or below
 * zero_rel * (the largest Ritz value) belong to the discrete null space
 * (gradient fields; for the central flux also its spurious modes of exactly
 * zero frequency) and are skipped; the next up to `nev` are returned.
 *   m         Lanczos steps, >= 2 (clipped to the number of E coefficients)
 *   nev       frequencies wanted, >= 1
 *   zero_rel  in [0, 1), e.g. 1e-8
 *   omega_out [nev] ascending frequencies (host); *nfound how many were filled
 *   resid_out [nev] (nullable) relative residual ||A u - th u||_M / (th ||u||_M)
 *             of each Ritz pair (th = omega^2, u its Ritz vector), computed on
 *             the device: small values mark converged frequencies
 * A degenerate eigenvalue is found once per Krylov direction it gains, so a
 * multiplicity is not resolved.  FP64 precision only (DGM_ERR_UNSUPPORTED
 * otherwise).  The fields are saved and restored.  Allocates (m + 4) x (number
 * of E coefficients) doubles of device memory (DGM_ERR_OOM if unavailable).
 * Blocks until the results are on the host. */
int dgm_resonances(dgm_problem* prob, int m, int nev, double zero_rel, double* omega_out, double* resid_out,
                   int* nfound);

/* Host-only helper of dgm_resonances (no device use): eigenvalues with indices
 * [i0, i1) in ascending order of the symmetric tridiagonal matrix with diagonal
 * d[k] and off-diagonal e[k-1] (e may be NULL for k = 1), by bisection on Sturm
 * counts, into vals[i1 - i0]; with vecs != NULL also unit eigenvectors
 * [i1 - i0][k] by inverse iteration.  DGM_ERR_INVALID_ARG unless
 * 0 <= i0 < i1 <= k. */
int dgm_tridiag_eig(int k, const double* d, const double* e, int i0, int i1, double* vals, double* vecs);

/* Launch-configuration autotuner of the per-step kernels (the time loop of
 * Sec. 3).  Each candidate configuration is timed (CUDA events, `steps` steps
 * after one warm-up step) on this problem's own fields with dt = 0, which
 * leaves the fields unchanged; the fastest is kept for all later calls.
 * Candidates: CUDA-core kernels (FP64, FP32) -- 4, 8, 16 or 24 blocks per SM;
 * with the central flux and variant 0 each also with the sparse curl, reported
 * as 1000 + blocks per SM (the dense and the sparse curl sum the same nonzero
 * products in different orders: fields then agree to round-off, not bitwise);
 * with the central flux, variant 0 or 3 and no compensated update also the
 * element-group kernels, reported as 2000 + blocks per SM (1 or 2, where that many
 * blocks' shared memory fits in an SM; the same sums as the sparse curl);
 * dense-operator tensor-core kernels (TC32, TC16X2, TC16 variant 1) -- 1 or 2 CTAs per
 * SM (2 only where the TMEM columns and shared memory of a CTA allow it);
 * resident-table tensor-core kernels (TC16, TCBF16) -- one configuration
 * (one CTA per SM), timed and reported like the others.  Candidates that differ
 * only in launch shape compute each element with the same operations, so the
 * fields of later runs do not depend on that choice; the energy's last bits can
 * (block partial sums).
 * Outputs (nullable): *ncand (<= DGM_AUTOTUNE_MAX), per candidate its
 * configuration value (blocks or CTAs per SM) and ms per step, and the index
 * of the chosen one.  Errors: DGM_ERR_INVALID_ARG for steps < 1. */
#define DGM_AUTOTUNE_MAX 12
int dgm_autotune(dgm_problem* prob, int steps, int* ncand, int* cand_config, double* cand_ms, int* chosen);

/* Point dipole current J(x, t) = dir delta(x - xs) f(t) with the zero-mean
 * pulse f(t) = -amp ((t - t0)/tau) exp(-((t - t0)/tau)^2): the E-equation of
 * Sec. 2 gains -(J, e), applied in every E-kick of dgm_run (and of the forward
 * runs of dgm_adjoint_grad) at the kick's midpoint time.  One source per
 * problem; amp = 0 removes it; dgm_kick applies no source.  xs must lie in the
 * mesh (DGM_ERR_INVALID_ARG otherwise). */
int dgm_set_source(dgm_problem* prob, const double* xs, const double* dir, double t0, double tau, double amp);
/* Time of the state: set by the caller, advanced by nsteps*dt in dgm_run. */
int dgm_set_time(dgm_problem* prob, double t);
int dgm_get_time(const dgm_problem* prob, double* t);

/* Replace the per-element eps and mu (> 0) of an existing problem; the fields
 * are kept.  Mass blocks of Sec. 3.3.1 scale with eps, mu. */
int dgm_set_materials(dgm_problem* prob, const double* eps, const double* mu);

/* Gradient of a field observable with respect to the per-element permittivity
 * and permeability by the discrete adjoint of the leapfrog (Sec. 3; central
 * flux):
 *   J = sum_{n=1..nsteps} sum_o |E^n(x_o)|^2,  x_o = xobs[o][0..2],
 * E^n the fields of dgm_run started from the current state.  The adjoint runs
 * the same E- and H-kicks backward in time (negative step) with point sources
 * 2 P^T P E^n; E^n and the staggered H^{n+1/2} are recomputed segment by
 * segment from checkpoints taken every ckpt_every steps.  dJdeps[nt] (host)
 * receives dJ/d eps_T, dJdmu[nt] (host, nullable) dJ/d mu_T (the H-kicks'
 * multipliers against the H increments, the opening half kick included),
 * J_out (host) J.  The state is restored.  Points must lie in the mesh.
 * Blocks; allocates. */
int dgm_adjoint_grad(dgm_problem* prob, double dt, int64_t nsteps, int nobs, const double* xobs,
                     int ckpt_every, double* J_out, double* dJdeps, double* dJdmu);

/* Batches: many independent problems on one device advanced together.  The
 * whole time loop of every run is captured once into a CUDA graph -- a fork,
 * one branch (stream) per run with all its phase kernels, a join -- so small
 * runs execute concurrently and the launch cost is paid once per call; the
 * graph is replayed while (nsteps, dt[], energy request, stream) stay the same.
 * dgm_batch_run: dt[nruns]; energy_out (nullable, host) [nruns][nsteps+1] as in
 * dgm_run.  Problems keep their own state, source and time; a problem must not
 * be used outside the batch while a batched run is in flight. */
typedef struct dgm_batch dgm_batch;
int dgm_batch_create(dgm_ctx* ctx, dgm_problem** probs, int nruns, dgm_batch** out);
int dgm_batch_destroy(dgm_batch* batch);
int dgm_batch_run(dgm_batch* batch, const double* dt, int64_t nsteps, void* stream, double* energy_out);

/* Per-kernel timing of one dgm_run_timed call: CUDA events recorded on the
 * launching stream around every phase kernel (summed, milliseconds) and the
 * number of kernels the call launched. */
typedef struct dgm_run_stats {
    double h_phase_ms;       /* H-phase kernels (incl. their fused energy partials) */
    double e_phase_ms;       /* E-phase kernels */
    double other_ms;         /* energy reductions */
    int64_t h_launches, e_launches, other_launches;
} dgm_run_stats;

/* dgm_run with per-kernel CUDA-event timing written to *stats (nullable). */
int dgm_run_timed(dgm_problem* prob, double dt, int64_t nsteps, void* stream,
                  double* energy_out, dgm_run_stats* stats);

/* Failure injection for tests of the bounded waits (tensor-core precisions
 * only; not part of the method of the paper).  The next `nlaunches` phase
 * kernels this problem launches each first wait on a barrier that nothing
 * arrives at; the wait gives up after about a millisecond, before the kernel
 * has issued any copy or MMA, the kernel records the timeout in the problem's
 * device error word, frees its tensor memory and returns without touching the
 * fields.  The host call that next reads the error word (dgm_run with
 * energies, dgm_run_composed, dgm_get_fields) returns DGM_ERR_TIMEOUT and
 * clears it; the problem stays usable.  nlaunches = 0 cancels a pending
 * injection.  DGM_ERR_UNSUPPORTED for the CUDA-core precisions, which have no
 * waits. */
int dgm_inject_wait_timeout(dgm_problem* prob, int nlaunches);

/* FP64 arithmetic peak of CUDA device `device` in TFLOP/s (2 flops per fused
 * multiply-add), measured with CUDA events over `repeats` timed launches of a
 * kernel of independent FMA chains that fills every SM (the best launch
 * counts).  The FP64 path's phase kernels are bound by FP64 arithmetic, so this
 * is their roofline denominator.  Not part of the method of the paper.
 * Allocates and frees a small device buffer; blocks. */
int dgm_measure_fp64_peak(int device, int repeats, double* tflops);

/* Discrete energy 1/2 (eps E,E) + 1/2 (mu H,H) [+ face term] of the current
 * state (no staggering), FP64. */
int dgm_energy(dgm_problem* prob, double* W);

/* The value of dgm_energy, written to *W_device (one double in device memory,
 * on the problem's device) and ordered on `stream`, without allocating any
 * device memory.  The paper has no counterpart; this serves callers that may
 * not call cudaMalloc/cudaFree (for example applications that hand all device
 * memory to their own pool at start-up).  Every precision is served: the
 * CUDA-core precisions through the H-phase kernel with dt = 0, the tensor-core
 * precisions through the state-energy kernel of the tiled state.  The partial
 * sums live in a fixed device array of 4096 doubles per device, shared by
 * every call: calls whose kernels overlap on the GPU race on it.  The first
 * call on a device looks up that array's address; make it before any stream
 * capture.  Problems needing more than 4096 partial sums are rejected with
 * DGM_ERR_INVALID_ARG; on GB300 (152 SMs) a problem uses at most 24 per SM
 * (CUDA-core precisions, autotuned) or 4 per SM (tensor-core precisions: two
 * CTAs, an E and an H sum each), so none is rejected there. */
int dgm_energy_noalloc(dgm_problem* prob, double* W_device, void* stream);

/* Initial data and evaluation (Sec. 2: initial conditions; covariant L2
 * projection, which for flat elements reduces to c_a = F^T sum_q w_q phi_a(xh_q)
 * u(x_q) / ||phi_a||^2 by Sec. 3.3.1).
 *
 * dgm_quad_rule: tensor Gauss-Legendre rule in the collapsed coordinates of the
 * reference tetrahedron with q1d points per direction (nq = q1d^3, exact for
 * polynomials of total degree <= 2 q1d - 3); xh [nq][3] reference points, w [nq]
 * weights summing to 1/6.  Any output may be NULL.  Needs no GPU.
 * dgm_element_maps: [nt][12] = X0 (3) and F row-major (9) of every element in
 * key order (Sec. 3.2.1).  Physical points are x = X0 + F xh.  Needs no GPU.
 * dgm_project_device: set E (and H) to the projections of point values
 * E_pts [nt][nq][3] (H_pts likewise, nullable) given at x = X0 + F xh_q of the
 * rule with q1d points.  Device pointers, FP64, ordered on `stream`.
 * dgm_eval_device: the reverse -- physical field values of the current E, H at
 * the same points (outputs nullable). */
int dgm_quad_rule(int q1d, int* nq, double* xh, double* w);
int dgm_element_maps(const dgm_mesh* mesh, double* out);
int dgm_project_device(dgm_problem* prob, int q1d, const double* E_pts, const double* H_pts,
                       void* stream);
int dgm_eval_device(dgm_problem* prob, int q1d, double* E_pts, double* H_pts, void* stream);

/* Host-array forms of the same, blocking:
 * dgm_quad_points: *count = nt * nq * 3; with xyz != NULL also the physical
 * points x = X0 + F xh_q of every element, [nt][nq][3] (computed on the device;
 * NULL xyz is a size query).
 * dgm_project: as dgm_project_device from host arrays [nt][nq][3] (one may be
 * NULL, not both).
 * dgm_eval: as dgm_eval_device into host arrays (one may be NULL, not both).
 * Each allocates and frees a device buffer of the arrays' size. */
int dgm_quad_points(dgm_problem* prob, int q1d, int64_t* count, double* xyz);
int dgm_project(dgm_problem* prob, int q1d, const double* E_pts, const double* H_pts);
int dgm_eval(dgm_problem* prob, int q1d, double* E_pts, double* H_pts);

/* Recurrences for the derivatives of the 3D shape functions (Sec. 3.2.2,
 * Sec. 4.2.2), host only, no GPU.  A relation in direction dir (0 x, 1 y, 2 z)
 *   sum_{s in SD} c_s d/d(dir) phi_{(i,j,k)+s} + sum_{s in S0} c_s phi_{(i,j,k)+s} = 0
 * ties shifts of the derivative to shifts of the functions.  For x the support
 * is the one printed in Sec. 4.2.2 (16 terms).  For y (20 terms) and z (19
 * terms) the paper states that relations exist but prints no support: these
 * were found by a numerical search.
 * dgm_grad_support: *nterms, the shifts [nterms][4] = (di, dj, dk, 1 if the term
 * carries the derivative else 0) (nullable), and *lead (nullable), the position
 * of the term that is highest in the order (degree, k, j, i).
 * dgm_grad_recurrence: the coefficients at every (i, j, k) with the shifted
 * indices <= p where the support carries a relation with a nonzero lead term:
 * all such indices for x and y, i >= 1 for z (d/dz of phi_0jk vanishes).  At
 * i >= 1 the relation is unique; at i = 0 there are several and the one with
 * the smallest coefficients (minimum norm) is returned.  Found numerically with the lead coefficient 1, in the printed
 * (unnormalised) basis;
 * *count relations, ijk [*count][3] and coef [*count][nterms] nullable for a
 * size query.  p in [1, 8].
 * dgm_grad_sweep: b [N3(p-1)] = coefficients of the derivative of
 * u = sum a_ijk phi_ijk (a [N3(p)], both lexicographic in (i, j, k),
 * unnormalised basis) by the backward sweep over those relations, visiting
 * indices by descending (degree, k, j, i).  Indices that lead no relation get
 * the dense column (exact quadrature).  *swept (nullable) counts the
 * coefficients a relation handled. */
int dgm_grad_support(int dir, int* nterms, int32_t* shifts, int* lead);
int dgm_grad_recurrence(int p, int dir, int* count, int32_t* ijk, double* coef);
int dgm_grad_sweep(int p, int dir, const double* a, double* b, int* swept);

/* Reference tables of the library (host, FP64, orthonormalised basis
 * phi_a / ||phi_a||), for inspection and tests:
 *   which = 0,1,2: D_x, D_y, D_z  [N3(p-1)][N3(p)], entry (b,a) = (d phi_a, phi_b)
 *   which = 3..6 : trace of face which-3  [N2(p)][N3(p)], entry (g,a) =
 *                  int psi_g(s,u) phi_a(face point) ds du, face basis orthonormal
 *   which = 7    : squared norms ||phi_a||^2 [N3(p)]
 * Needs no GPU.  `count` = capacity of `out` in doubles; the required size is
 * returned in *needed. */
int dgm_reference_table(int p, int which, double* out, int64_t count, int64_t* needed);

/* Reference tables of the 2D triangle solver (host, FP64, orthonormalised
 * Dubiner basis psi_a / ||psi_a|| of Eq. (4) on the reference triangle with
 * vertices (0,0), (1,0), (0,1)).  The 2D TE fields: E in the plane of degree p,
 * H along z of degree p - 1 (Sec. 2's pair of spaces in two dimensions); the
 * derivative tables are those whose sparsity the printed 2D relations of
 * Sec. 4.2.1 describe, the traces those of Sec. 3.2.3 on edges:
 *   which = 0,1  : D_x, D_y  [N2(p-1)][N2(p)], entry (b,a) = (d psi_a, psi_b)
 *   which = 2..4 : E trace on edge which-2  [p+1][N2(p)], entry (g,a) =
 *                  int_0^1 psi_a(edge point at s) L_g(s) ds
 *   which = 5..7 : H trace on edge which-5  [p][N2(p-1)], the same
 *   which = 8    : squared norms ||psi_a||^2 [N2(p)]
 * Edge f is opposite reference vertex f, parametrised from its lower-numbered
 * vertex to its higher one; L_g = sqrt(2g+1) P_g(2s-1), orthonormal on [0,1].
 * Needs no GPU.  `count` = capacity of `out` in doubles; the required size is
 * returned in *needed.  Errors: DGM_ERR_INVALID_ARG for p outside [1, DGM_PMAX],
 * `which` out of range or `out` too small. */
int dgm_reference_table_2d(int p, int which, double* out, int64_t count, int64_t* needed);

/* 2D triangle solver (TE fields).  E = (E_x, E_y) in the plane, covariant of
 * degree p: E|_T(x) = F^{-T} sum_a c_{m,a} e_m psi_a(Phi^{-1} x), m = 0, 1, with
 * psi the printed (unnormalised) Dubiner basis of Eq. (4), multi-indices (i,j),
 * i+j <= p, lexicographic with i outermost; H = H_z scalar of degree p - 1:
 * H|_T(x) = sum_b d_b psi_b(Phi^{-1} x).  The triangle's vertices are ordered by
 * ascending key (vertex_key[v] if given, else v), Phi(xh) = X0 + F xh,
 * F = [X1-X0, X2-X0].  The scheme is the central-flux system of Sec. 2.1 for
 * these fields (eps dE/dt = curl H, mu dH/dt = -curl E, curl E = d_x E_y - d_y E_x,
 * curl H = (d_y H, -d_x H)), with the leapfrog of Sec. 3:
 *   d/dt (eps E, e)_T = (H, curl e)_T - ({{H}}, n x e)_dT
 *   d/dt (mu H, h)_T  = -(curl E, h)_T + (1/2 n x [[E]], h)_dT
 * n x v = n_x v_y - n_y v_x, [[E]] = E_T - E_nbr, {{H}} = (H_T + H_nbr)/2; edges
 * without a partner are PEC walls (ghost E_nbr = -E_T tangentially, H_nbr = H_T);
 * two edges whose two keys coincide are glued (periodic).  FP64 or FP32
 * (`precision` DGM_PREC_FP64 / DGM_PREC_FP32; else DGM_ERR_UNSUPPORTED).
 * Layouts (host arrays, FP64): E [nt][2][N2(p)], H [nt][N2(p-1)].
 * Errors of create: DGM_ERR_INVALID_ARG for ids out of range, repeated keys in
 * one triangle, degenerate triangles (|det F| <= 1e-12 (max edge component)^2),
 * edges shared by more than two triangles, a triangle glued to itself,
 * non-positive eps or mu, p outside [1, DGM_PMAX]. */
typedef struct dgm_problem2d dgm_problem2d;
/* Edge counts of a 2D triangle mesh with the adjacency dgm_problem2d_create
 * builds (keys, periodic gluing, PEC boundary): *nedges distinct edges, of which
 * *nboundary have no partner.  Host only, no GPU; the same argument checks and
 * errors as dgm_problem2d_create (eps = mu = 1). */
int dgm_mesh2d_info(int64_t nv, const double* xy, int64_t nt, const int32_t* tris, const int32_t* vertex_key,
                    int64_t* nedges, int64_t* nboundary);
int dgm_problem2d_create(dgm_ctx* ctx, int64_t nv, const double* xy, int64_t nt, const int32_t* tris,
                         const int32_t* vertex_key, int p, const double* eps, const double* mu, int precision,
                         dgm_problem2d** out);
int dgm_problem2d_destroy(dgm_problem2d* prob);
/* Lengths (in doubles) of the canonical E and H arrays. */
int dgm_problem2d_sizes(const dgm_problem2d* prob, int64_t* nE, int64_t* nH);
int dgm_set_fields2d(dgm_problem2d* prob, const double* E, const double* H);
int dgm_get_fields2d(dgm_problem2d* prob, double* E, double* H);
/* One half of the symplectic Euler step: which = 0 advances H by dt from the
 * current E, which = 1 advances E by dt from the current H. */
int dgm_kick2d(dgm_problem2d* prob, int which, double dt);
/* nsteps leapfrog steps with the opening and closing half kicks of H, as
 * dgm_run; energy_out (nullable, nsteps + 1 values) receives the modified energy
 * W^n = 1/2 (eps E^n, E^n) + 1/2 (mu H^{n-1/2}, H^{n+1/2}), n = 0..nsteps. */
int dgm_run2d(dgm_problem2d* prob, double dt, int64_t nsteps, void* stream, double* energy_out);

#ifdef __cplusplus
}
#endif

#endif /* DGM_H */
