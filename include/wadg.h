/*
 * wadg.h -- C ABI of the GB300 weight-adjusted DG (WADG) library.
 *
 * Method: Chan, Hewett & Warburton, "Weight-adjusted discontinuous Galerkin
 * methods: curvilinear meshes" (arXiv:1608.03836).  The library evaluates the
 * semi-discrete acoustic system dQ/dt = -M~^{-1} A_h Q (Sec. 4) on curved
 * tetrahedral meshes with the strong-weak formulation (Sec. 4.1), the
 * weight-adjusted mass inverse M^^{-1} M_{c^2/J} M^^{-1} applied matrix-free as
 * P_q diag(c^2_q/J_q) V_q (Sec. 6.2, Eq. (matfree); Sec. 7 for c^2), and the
 * five-stage fourth-order low-storage Runge-Kutta scheme (Sec. 5.2).
 *
 * Conventions shared by every entry point
 *  - Returns a wadg_status code; nothing aborts, traps or exits.  Argument and
 *    geometry errors are detected on the host before any launch.  After an
 *    error, wadg_last_error(mesh) holds a one-line description.
 *  - Reference element: {r,s,t >= -1, r+s+t <= -1}, vertices v0=(-1,-1,-1),
 *    v1=(1,-1,-1), v2=(-1,1,-1), v3=(-1,-1,1); faces f0=(v0,v1,v2),
 *    f1=(v0,v1,v3), f2=(v1,v2,v3), f3=(v0,v2,v3).
 *  - Nodal layout ("lattice"): the solution is stored as values at the
 *    equispaced degree-N lattice, node (i,j,k), i+j+k <= N, at
 *    (-1+2i/N, -1+2j/N, -1+2k/N), ordered i fastest, then j, then k.
 *    Np = (N+1)(N+2)(N+3)/6.
 *  - Field buffers Q, res, dQdt are caller-owned DEVICE arrays laid out
 *    [4][K][S][Np] (fields p, u1, u2, u3; element; shot; node), in the mesh
 *    precision (double for WADG_FP64, float otherwise), 16-byte aligned.
 *  - Volume quadrature: collapsed Gauss-Jacobi rule with N+1 points per
 *    direction (exact to degree 2N+1, Sec. 6.2), Nq = (N+1)^3; point
 *    (ia,ib,ic) has index ia + (N+1)(ib + (N+1) ic), with
 *    r = (1+a)(1-b)(1-c)/4 - 1, s = (1+b)(1-c)/2 - 1, t = c and a, b, c the
 *    ascending Gauss-Jacobi nodes for the weights 1, (1-b), (1-c)^2.
 *  - Face quadrature: collapsed rule with N+1 points per direction on the
 *    reference triangle, Nfq = (N+1)^2.  A face shared by two elements is
 *    integrated by both at the points of its owner, the element with the lower
 *    index (Sec. 6.4 uses values at the same "neighbouring" face points).
 *  - Streams are passed as opaque pointers (cudaStream_t; NULL = legacy
 *    default stream).  Work is enqueued; no entry point synchronises unless it
 *    returns a host value (wadg_energy, wadg_l2_error).
 */
#ifndef WADG_H
#define WADG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wadg_mesh wadg_mesh;  /* opaque, library-owned */
typedef void* wadg_stream;           /* a cudaStream_t */

enum wadg_status {
    WADG_OK = 0,
    WADG_EINVAL = -1,       /* bad argument (size, pointer, alignment)        */
    WADG_ENOMEM = -2,       /* device or host allocation failed               */
    WADG_ECUDA = -3,        /* a CUDA call failed (message in last_error)     */
    WADG_EGEOM = -4,        /* J <= 0, inverted element or non-conforming face */
    WADG_ESTATE = -5,       /* call order (e.g. operators not set)            */
    WADG_ETIMEOUT = -6,     /* a bounded device wait expired                  */
    WADG_EUNSTABLE = -7,    /* non-finite energy                              */
    WADG_EUNSUPPORTED = -8  /* order or precision not built                   */
};

enum wadg_precision {
    WADG_FP64 = 0,          /* FP64 fields, FP64 arithmetic (CUDA cores)      */
    WADG_FP32 = 1,          /* FP32 fields, FP32 arithmetic (CUDA cores)      */
    WADG_FP32_TF32 = 2,     /* FP32 fields; the dense products of the stage on
                               the tensor cores in tf32 (one product, 10-bit
                               mantissa operands, FP32 accumulation); N <= 5
                               (N = 5 on the collapsed 216-point or the
                               96-point volume rule) and
                               K * shots * Np < 2^31.  About 1e-3 relative
                               on the RHS.  Adjoint and diagnostics as
                               WADG_FP32. */
    WADG_FP32_3XBF16 = 3    /* FP32 fields; the dense products of the stage on
                               the tensor cores with split bf16 operands
                               (hi*hi + hi*lo + lo*hi, FP32 accumulation);
                               N <= 5 (N = 5 on the collapsed 216-point or
                               the 96-point volume rule) and
                               K * shots * Np < 2^31.  Adjoint
                               and diagnostics as WADG_FP32. */
};

/* Library version as major*10000 + minor*100 + patch. */
int wadg_version(void);

/* Create a mesh (Sec. 2: elements D^k = Phi^k(D^), isoparametric of degree N).
 *   N        polynomial degree, 1 <= N <= 6.
 *   VXYZ     host [Nv][3] vertex coordinates (FP64).
 *   EToV     host [K][4] vertex indices; each element must be positively
 *            oriented for the reference vertex order above (WADG_EGEOM if not).
 *   geom_xyz host [K][Np][3] physical coordinates of each element's lattice
 *            nodes (the isoparametric map is their degree-N interpolant), or
 *            NULL for straight-sided (affine) elements.
 *   out      receives the handle.
 * Builds connectivity (faces matched by their vertex triples; a face shared by
 * more than two elements is WADG_EGEOM), the reference operators, and the FP64
 * geometric factors on the current CUDA device: J and G_ai = J dx^_a/dx_i at
 * volume points and n J^f at face points (Sec. 4.1: these are polynomial for
 * an isoparametric map).  WADG_EGEOM if J <= 0 at any volume point.  The
 * library copies what it needs; the caller keeps ownership of its arrays. */
int wadg_mesh_create(int N, int64_t Nv, const double* VXYZ, int64_t K, const int64_t* EToV,
                     const double* geom_xyz, wadg_mesh** out);

/* wadg_mesh_create with an explicit volume rule: nq points
 * rule[q] = (r, s, t, w) on the reference tetrahedron (vertices (-1,-1,-1),
 * (1,-1,-1), (-1,1,-1), (-1,-1,1); weights positive, summing to its volume
 * 4/3), used for the volume terms, the weight-adjusted update, the
 * geometric factors, c^2 and the diagnostics; the face rule stays the
 * collapsed one.  It must be exact to degree 2N (checked: P_q V_q = I,
 * WADG_EUNSUPPORTED otherwise) and should be exact to 2N+1 (Sec. 4, Sec. 6.2).
 * The stage kernels are built for nq = (N+1)^3 and for the fewer-point
 * symmetric rules with nq = 14 (N = 2), 35 (N = 3), 63 (N = 4) and 96
 * (N = 5); other sizes are WADG_EUNSUPPORTED.  With the fewer-point sizes
 * the strong formulations, the adjoint and WADG_FP32 batches are not
 * available (WADG_EUNSUPPORTED / WADG_ESTATE); tensor-core batches are.
 * rule = NULL is wadg_mesh_create. */
int wadg_mesh_create_rule(int N, int64_t Nv, const double* VXYZ, int64_t K, const int64_t* EToV,
                          const double* geom_xyz, int nq, const double* rule, wadg_mesh** out);

/* Select precision and material, and allocate the library's work buffers.
 *   precision WADG_FP64 or WADG_FP32.
 *   shots     S >= 1 right-hand sides sharing the mesh (columns [K][S]).
 *   tau_p, tau_u  penalty parameters of the strong-weak flux (Sec. 4.1;
 *             1 = upwind, 0 = central), both >= 0.
 *   c2q       host [K][Nq] values of c^2 at the volume quadrature points
 *             (Sec. 7), or NULL for c^2 = 1; every value must be > 0.
 * May be called again to change any of these. */
int wadg_set_operators(wadg_mesh* mesh, int precision, int shots, double tau_p, double tau_u,
                       const double* c2q);

/* Status of the device-side checks: synchronises `stream` and returns
 * WADG_ETIMEOUT if a bounded wait inside a tensor-core kernel expired since
 * the last call (the flag is then cleared), WADG_OK otherwise. */
int wadg_device_status(wadg_mesh* mesh, wadg_stream stream);

/* Test hook for the failure path of the bounded device waits (no fault, trap
 * or hang is involved): launches one block that waits, with the same bounded
 * loop as the tensor-core kernels, max_iters times (1 .. 2^22) on an mbarrier
 * that nothing arrives at.  The expired wait sets the device error flag, so
 * the next wadg_device_status returns WADG_ETIMEOUT. */
int wadg_selftest_bounded_wait(wadg_mesh* mesh, uint32_t max_iters, wadg_stream stream);

/* Sizes: info[0..7] = N, K, Np, Nq, Nfp, Nfq, S, precision (S, precision are
 * -1 before wadg_set_operators). */
int wadg_mesh_info(const wadg_mesh* mesh, int64_t info[8]);

/* Physical coordinates of the volume quadrature points, host [K][Nq][3] FP64. */
int wadg_volume_points(const wadg_mesh* mesh, double* xyz);

/* Reference rules for degree N (host only, no device work): rst_q [Nq][3],
 * w_q [Nq], rs_f [Nfq][2], w_f [Nfq].  Any pointer may be NULL. */
int wadg_reference_rules(int N, double* rst_q, double* w_q, double* rs_f, double* w_f);

/* Weight-adjusted pseudo-projection P_N u = Pi_N(J^{-1} Pi_N(u J)) (Sec. 3,
 * Theorem) of values at the volume quadrature points.
 *   fq  device [4][K][S][Nq] FP64 values of (p, u1, u2, u3).
 *   Q   device [4][K][S][Np] output in the mesh precision. */
int wadg_project(wadg_mesh* mesh, const double* fq, void* Q, wadg_stream stream);

/* Right-hand side dQdt = -M~^{-1} A_h Q (Sec. 4; strong-weak A_h of Sec. 4.1;
 * M~^{-1} = P_q diag(W) V_q M^^{-1}, W = c^2/J for p and 1/J for u, Sec. 6.2
 * and Sec. 7).  Q and dQdt are device [4][K][S][Np] and must not overlap. */
int wadg_rhs(wadg_mesh* mesh, const void* Q, void* dQdt, wadg_stream stream);

/* nsteps steps of LSRK(5,4) (Sec. 5.2) from time t0 with step dt.  Each stage:
 * res = a_s res + dt (-M~^{-1} A_h Q + source); Q = Q + b_s res.
 *   Q, res   device [4][K][S][Np], updated in place.  The first stage has
 *            a_1 = 0, so the incoming res is not read (a step does not depend
 *            on it); on return res holds the last stage's residual.
 *   traces   device [nsteps][S][R] in the mesh precision: pressure at the
 *            receivers after every step, or NULL (ignored when R = 0).
 * Sources and receivers are those set by wadg_set_sources/wadg_set_receivers. */
int wadg_step(wadg_mesh* mesh, void* Q, void* res, double t0, double dt, int nsteps, void* traces,
              wadg_stream stream);

/* Formulation of the stage (Sec. 4.1): 0 = strong-weak (the default; the
 * pressure equation integrated by parts once); 1 = strong (both equations
 * integrated by parts twice: volume term -int (div u) v, surface term
 * -int 1/2 ([u].n - tau_p [p]) v), with its volume and surface terms on
 * collapsed rules of max(N+1, 2N-1) and 2N points per direction, exact for
 * the degree 4N-3 volume and 4N-2 surface integrands of an isoparametric map,
 * so that it is energy stable (Sec. 4.1, Sec. 6.3); 2 = the strong form on
 * the degree 2N+1 rules of the strong-weak form (under-integrated on curved
 * elements; faster, stability not guaranteed, Sec. 6.5).  The weight-adjusted
 * update always uses the degree 2N+1 volume rule.  Form 1 computes and keeps
 * the geometric factors at its rules' points (9 values per volume point, 3
 * per face point, in the mesh precision); it returns WADG_EGEOM if J <= 0 at
 * one of them.  The strong forms are built for the CUDA-core precisions and
 * N <= 5, for wadg_rhs, wadg_step, wadg_step_host and wadg_solve; the adjoint
 * and batches require form 0.  WADG_EUNSUPPORTED otherwise.  May be called
 * before or after wadg_set_operators; on failure the previous formulation
 * stays in effect. */
int wadg_set_formulation(wadg_mesh* mesh, int form);

/* Update weights (Sec. 3, the remark after the moment estimate): 0 = the
 * pointwise weights W_p = c^2/J, W_u = 1/J at the volume points (the default,
 * Sec. 6.2, Sec. 7); 1 = locally conservative weights W_p = 1 / Pi_N(J/c^2),
 * W_u = 1 / Pi_N(J), the mass weights projected onto P^N with the volume rule
 * (FP64, once), so that every element's update conserves its zeroth moment:
 * sum_q w_q (J/c^2)_q dp/dt(x_q) equals the load functional at v = 1 (and
 * likewise for u with J).  Applies to every precision and formulation
 * (tensor cores included: the weights are part of the geometric factors).
 * May be called before or after wadg_set_operators (which recomputes the
 * weights when c^2 changes).  WADG_EGEOM if a projected weight is not
 * positive at a volume point (the previous setting stays in effect).  The c^2
 * gradient of the adjoint (wadg_step_record / wadg_step_adjoint with ystore)
 * is built for the pointwise weights: WADG_EUNSUPPORTED under 1. */
int wadg_set_conservation(wadg_mesh* mesh, int on);

/* Compensated summation of the state in the LSRK steps (FP32 fields; not in
 * the paper): each stage adds b res to Q together with the rounding error
 * carried from the previous stages (Fast2Sum into a mesh-owned [4][K][S][Np]
 * float buffer, the carry), so the FP32 state no longer loses 2^-24 of its
 * value per stage.  on = 1: the carry is cleared at the start of every
 * wadg_step / wadg_solve / wadg_step_host call (a call's result depends on
 * its inputs only); on = 2: the carry is kept from one call to the next, so
 * that a run split into several calls equals one call bit for bit (clear it
 * by calling wadg_set_compensation again, or save and restore it with
 * wadg_compensation_carry beside a checkpoint of Q and res, when the state
 * is replaced between calls); 0 = plain FP32 updates (the default).  Every
 * call with on != 0 clears the carry (synchronously).  The stage's
 * right-hand side reads Q only.  Costs one read and one write of the carry
 * per stage.  WADG_EUNSUPPORTED for WADG_FP64 (wadg_set_operators with
 * WADG_FP64 turns it off); mesh batches and the adjoint entry points refuse
 * compensated meshes (WADG_ESTATE); WADG_EINVAL for other values of on. */
int wadg_set_compensation(wadg_mesh* mesh, int on);

/* The compensation carry to (direction 0) or from (direction 1) lo, a host
 * or device buffer of 4 K S Np floats (the layout of Q), for checkpoints of
 * compensated runs (on = 2).  Enqueued on stream; returns after the copy has
 * completed.  WADG_ESTATE when compensation is off; WADG_EINVAL for a null
 * buffer or another direction. */
int wadg_compensation_carry(wadg_mesh* mesh, void* lo, int direction, wadg_stream stream);

/* Planar and curved elements in separate tensor-core kernels (Sec. 6: planar
 * elements admit a cheaper implementation; N <= 5): an element is affine when
 * its geometry nodes are its vertices' affine lattice map (to 1e-13 of its
 * extent; every element when wadg_mesh_create got no nodes).  A tile of 128
 * columns whose elements are all affine may run a kernel that reads each
 * element's constant geometric factors and normals once instead of at every
 * quadrature point (the update weights c^2/J stay per point); the curved
 * kernel runs the other tiles, one launch after the other in the stage.
 * on = 1 (the default) plans the split from the tile counts: the planar
 * launch takes the all-affine tiles less those that would open a partial
 * round of its CTAs, and only when the rounds saved outweigh a second
 * launch (so meshes of fewer tiles than SMs stay on one launch); on = 2 runs
 * every all-affine tile on the planar kernel; on = 0 runs every tile on the
 * curved kernel.  Results equal the curved kernel's to rounding.  The lists
 * are built by wadg_set_operators (tensor-core precisions).  WADG_EINVAL for
 * other values of on. */
int wadg_set_planar_split(wadg_mesh* mesh, int on);

/* info[0..3] = affine elements, tiles of affine elements, tiles, tiles the
 * planar kernel runs (the last three are 0 until wadg_set_operators selects
 * a tensor-core precision with N <= 5 and some tile is all affine). */
int wadg_planar_info(const wadg_mesh* mesh, int64_t info[4]);

/* wadg_step on host fields: Q and res are HOST [4][K][S][Np] arrays in the
 * mesh precision (pinned memory gives the fastest copies).  Q is copied to a
 * device buffer owned by the mesh, stepped nsteps times, and Q and res are
 * copied back before the call returns (the call waits for the stream).  The
 * incoming res is not copied: a step does not read it (a_1 = 0, see
 * wadg_step).  res may be NULL: the residual is then kept on the device and
 * not returned (only the state Q crosses the link).  nsteps = 0 leaves both
 * unchanged.  No receiver traces. */
int wadg_step_host(wadg_mesh* mesh, void* Q, void* res, double t0, double dt, int nsteps, wadg_stream stream);

/* Solve from t0 to t0 + T (Sec. 5.2 time stepping): nsteps = ceil(T/dt_max)
 * LSRK(5,4) steps of dt = T/nsteps, exactly the launches of wadg_step.  All
 * launches of the solve are captured once into a CUDA graph on a library
 * stream and replayed; the graph is kept in the mesh and reused while Q, res,
 * traces, t0, dt, nsteps and the operators, sources and receivers are
 * unchanged.  The work is ordered after the caller's earlier work on `stream`
 * and before its later work (events); the call does not synchronise.
 *   traces      device [nsteps][S][R] or NULL.
 *   nsteps_out  host int receiving nsteps, or NULL. */
int wadg_solve(wadg_mesh* mesh, void* Q, void* res, double t0, double T, double dt_max, void* traces,
               int* nsteps_out, wadg_stream stream);

/* Point sources, one per shot: a Ricker wavelet (1-2 pi^2 f0^2 tau^2)
 * exp(-pi^2 f0^2 tau^2), tau = t - t0, times delta(x - x_s) added to the
 * pressure equation at every stage time.
 *   xyz  host [S][3] physical source positions (S = shots); NULL removes the
 *        sources.  A point outside the mesh is WADG_EINVAL. */
int wadg_set_sources(wadg_mesh* mesh, const double* xyz, double f0, double t0);

/* Receivers: R points per shot, host [S][R][3]; R = 0 removes them. */
int wadg_set_receivers(wadg_mesh* mesh, int R, const double* xyz);

/* Energy 1/2 int (p^2/c^2 + |u|^2) by the volume rule, summed over shots,
 * FP64 reduction; E is a host double.  WADG_EUNSTABLE if not finite. */
int wadg_energy(wadg_mesh* mesh, const void* Q, double* E, wadg_stream stream);

/* The energy of wadg_energy, computed without allocating anything.  The paper
 * has no counterpart: this entry point serves callers that must not call
 * cudaMalloc when they need the value -- code inside a framework whose caching
 * allocator owns the device memory budget, and real-time loops that must not
 * wait on the driver's allocator.  Like wadg_energy it returns E on the host,
 * so it synchronises `stream` before returning.  Its scratch is a fixed array of 2^20 + 1 doubles
 * (8 MiB) in device memory that every GPU loading the library holds until the
 * process exits; a mesh with K*S > 2^20 columns is rejected with WADG_EINVAL.
 * The first call on a device looks up the array's address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array, so calls that
 * overlap on the GPU (other streams, other host threads) race and return wrong
 * values; every slot a call reads it writes first, so nothing needs clearing.
 * Q, E, stream and the return codes are as for wadg_energy. */
int wadg_energy_noalloc(wadg_mesh* mesh, const void* Q, double* E, wadg_stream stream);

/* L2 error sqrt(sum_k int (q_h - q)^2) over the fields in field_mask (bit f for
 * field f) against exact values at the volume points, device [4][K][S][Nq]
 * FP64.  err is a host double. */
int wadg_l2_error(wadg_mesh* mesh, const void* Q, const double* exact_q, int field_mask, double* err,
                  wadg_stream stream);

/* ---- Discrete adjoint (gradients of receiver misfits) -------------------
 * The paper has no adjoint; these entry points apply the exact transposes of
 * the discrete operators above: the strong-weak load operator A_h (Sec. 4.1),
 * the weight-adjusted update P_q diag(W) V_q M^^{-1} (Sec. 6.2, Eq. (matfree);
 * Sec. 7) and the LSRK(5,4) stage recurrence (Sec. 5.2).  With L the operator
 * of wadg_rhs, the reverse of stage s is mu = lam_res + b_s lam_Q,
 * lam_Q += dt L^T mu, lam_res = a_s mu. */

/* out = L^T lambda (transpose of wadg_rhs).  lambda, out device [4][K][S][Np],
 * distinct, mesh precision. */
int wadg_rhs_adjoint(wadg_mesh* mesh, const void* lambda, void* out, wadg_stream stream);

/* One LSRK step exactly as wadg_step with nsteps = 1 that also records, for
 * each of its 5 stages, y_q = (V_q M^^{-1} b_p)_q / J_q at the volume points
 * (the factor by which the pressure update depends on c^2_q).
 *   ystore  device [5][K][S][Nq] in the mesh precision, or NULL (no record).
 *   traces  device [S][R] receiver pressures after the step, or NULL. */
int wadg_step_record(wadg_mesh* mesh, void* Q, void* res, double t0, double dt, void* ystore, void* traces,
                     wadg_stream stream);

/* Reverse of one LSRK step.  lamQ, lamR (device [4][K][S][Np], distinct) hold
 * the adjoints of Q and res after the step and are replaced by those before
 * it.  ystore: the record of the same step from wadg_step_record, or NULL;
 * dc2: device [K][Nq] FP64 accumulator of dJ/dc^2_q (summed over shots),
 * NULL exactly when ystore is NULL. */
int wadg_step_adjoint(wadg_mesh* mesh, void* lamQ, void* lamR, double dt, const void* ystore, double* dc2,
                      wadg_stream stream);

/* Transpose of the receiver samples: lamQ[p] += sum_r w_r l(x^_r) in each
 * receiver's column.  weights device [S][R] in the mesh precision. */
int wadg_receivers_adjoint(wadg_mesh* mesh, const void* weights, void* lamQ, wadg_stream stream);

/* The reverse of one checkpoint segment of nsteps steps in a single call:
 * when ystore is given, the segment is first recomputed forward from its
 * checkpoint as by wadg_step_record, recording every step's stage factors;
 * then, for n = nsteps - 1 .. 0, the receiver adjoint of step n's weights
 * (as wadg_receivers_adjoint) followed by the reverse of step n (as
 * wadg_step_adjoint).  The same kernels in the same order as those calls.
 *   Q, res   device [4][K][S][Np]: the state (Q, res) at t0 (the segment's
 *            start); advanced to t0 + nsteps dt by the recompute.  Read only
 *            when ystore is given (the adjoint of the linear steps does not
 *            depend on the state); may then be NULL.
 *   weights  device [nsteps][S][R] in the mesh precision, dJ/d(trace) of the
 *            segment's steps, or NULL (no receiver terms).
 *   lamQ, lamR  adjoints after the segment, replaced by those before it.
 *   ystore   device [nsteps][5][K][S][Nq] scratch in the mesh precision, or
 *            NULL; dc2 device [K][Nq] FP64 accumulator, NULL exactly when
 *            ystore is NULL. */
int wadg_segment_adjoint(wadg_mesh* mesh, void* Q, void* res, double t0, double dt, int nsteps,
                         const void* weights, void* lamQ, void* lamR, void* ystore, double* dc2,
                         wadg_stream stream);

/* ---- Batches of meshes of uneven size and degree -------------------------
 * Not in the paper, which tunes the number of elements per work-group for
 * each kernel (Sec. 6.1) but steps one mesh at a time.  A batch steps several
 * meshes together, with exactly the arithmetic of wadg_step per mesh
 * (results are bitwise equal):
 *   - WADG_FP32 meshes: each LSRK stage is ONE persistent launch over a work
 *     list of (mesh, tile) items, heaviest degree first;
 *   - tensor-core meshes (all WADG_FP32_3XBF16 or all WADG_FP32_TF32, N <= 5):
 *     the meshes of one class (same degree, volume rule, shots and
 *     penalties) are stepped as one combined mesh (their elements in
 *     sequence, the geometry copied into one interleaved table at creation),
 *     one tensor-core launch per class and stage, so that tiles of small
 *     meshes share the SMs; each step call copies the members' fields into
 *     the combined buffers and back (device to device).  The geometry is
 *     taken at creation: a batch made before a member's operators or
 *     conservation setting change keeps the old ones.
 * Point sources and receivers are not applied in batch stepping (a
 * tensor-core batch refuses meshes that have them: WADG_ESTATE).
 * Q[i], res[i]: device [4][K_i][S_i][Np_i] float buffers of mesh i. */
typedef struct wadg_batch wadg_batch;

/* meshes: host array of `count` handles on the same device, all set to
 * WADG_FP32 or all to the same tensor-core precision (WADG_ESTATE
 * otherwise).  The batch keeps the handles (not owned); destroy it before
 * the meshes.  A mesh whose precision or shots change afterwards makes the
 * stepping calls return WADG_ESTATE. */
int wadg_batch_create(wadg_mesh* const* meshes, int count, wadg_batch** out);

/* info[0..4] = meshes, work items, persistent blocks in use, largest
 * resident grid (occupancy x SMs) for the tile rule in use, the tile rule in
 * use (0, 1 or 2; see wadg_batch_autotune).  Tensor-core batches: meshes,
 * 128-column tiles over all classes, SMs, SMs, -1 (one schedule; the grid,
 * rule and autotuner calls have no effect on them). */
int wadg_batch_info(const wadg_batch* batch, int64_t info[5]);

/* Number of persistent blocks (clamped to the number of work items). */
int wadg_batch_set_grid(wadg_batch* batch, int grid);

/* Tile rule (0, 1 or 2; WADG_EINVAL otherwise), as wadg_batch_autotune
 * describes them; the grid is clamped to the rule's work items.  A captured
 * solve is captured again with the new rule or grid on its next call. */
int wadg_batch_set_rule(wadg_batch* batch, int rule);

/* Autotuner: for each of three tile rules, times right-hand-side launches of
 * the whole batch with 1, 2, 3, 4, 6, 8 blocks per SM (as occupancy allows)
 * and one block per item; keeps the fastest rule and grid and returns the
 * grid in grid_out (nullable).  The rules (one kernel holds every degree, so
 * its registers are the largest degree's and its shared memory the largest
 * tile's):
 *   0: the single-mesh columns per tile, registers capped for 2 blocks per SM;
 *   1: the same tiles, registers capped for 3 blocks per SM;
 *   2: tiles of at most 56 KB, registers capped for 4 blocks per SM.
 * Q and res are not modified; each mesh's work buffer is overwritten.
 * Synchronises `stream`.  Every rule gives bitwise the results of wadg_step:
 * every column's products are accumulated in the same order whatever the
 * tile width. */
int wadg_batch_autotune(wadg_batch* batch, void* const* Q, void* const* res, int* grid_out, wadg_stream stream);

/* nsteps LSRK(5,4) steps of every mesh (5 launches per step in total). */
int wadg_batch_step(wadg_batch* batch, void* const* Q, void* const* res, double t0, double dt, int nsteps,
                    wadg_stream stream);

/* As wadg_solve for the whole batch: the launches of the solve are captured
 * once into a CUDA graph, kept and replayed while the buffers, t0, dt and
 * nsteps are unchanged. */
int wadg_batch_solve(wadg_batch* batch, void* const* Q, void* const* res, double t0, double T, double dt_max,
                     int* nsteps_out, wadg_stream stream);

void wadg_batch_destroy(wadg_batch* batch);
const char* wadg_batch_last_error(const wadg_batch* batch);

void wadg_mesh_destroy(wadg_mesh* mesh);
const char* wadg_status_string(int status);
const char* wadg_last_error(const wadg_mesh* mesh);

#ifdef __cplusplus
}
#endif
#endif /* WADG_H */
