/*
 * dwos.h - C ABI of the GB300 (sm_103a) differential walk-on-spheres library.
 *
 * The library estimates, at chosen query points x of a domain Omega whose
 * boundary Gamma is a 2D polyline or a 3D triangle mesh,
 *   - the solution u(x) of the screened Poisson Dirichlet problem
 *         -Lap u + sigma u = f  in Omega,   u = g  on Gamma
 *     by walk on spheres (Miller et al., "Differential Walk on Spheres",
 *     TOG 2024: Eq. (bvp) of Sec. 3.2, the estimator Eq. (wos) and Algorithm 1
 *     of Sec. 3.3, Russian roulette as in Sec. 3.3; each step's ball has
 *     radius d(x) - 1e-3 eps, a clearance that keeps FP32 landing points on
 *     the domain's side of the boundary; any ball inside the domain gives an
 *     unbiased step);
 *   - its derivative udot = du/dtheta with respect to every shape and
 *     boundary-data parameter theta in R^N, by differential walk on spheres
 *     (Eq. (bvp_deriv) of Sec. 4.1, the estimator Eq. (wos_deriv) and
 *     Algorithm 2, with the backward-difference normal derivative of
 *     Eq. (dudn_fd_estimate) and the nested forward walks it launches from
 *     the offset point xbar - h n);
 *   - reverse-mode derivatives of the squared loss over the query points with
 *     the U-statistic product estimator (Sec. 4.3, Eqs. (squared_loss_deriv)
 *     and (ustatistics)), and vector-Jacobian products with a given cotangent.
 *
 * Sign of the source: Eq. (bvp) is printed as Lap u - sigma u = f, but
 * Algorithm 1 adds +G f / p with the positive ball Green's function; this
 * library follows the algorithm, so f is the source of -Lap u + sigma u = f.
 *
 * Conventions
 *  - Every call returns a dwos_status.  On error nothing is written to the
 *    outputs and dwos_last_error() describes the cause.
 *  - Pointers are host or device memory as the call's `mem` flag says
 *    (DWOS_MEM_HOST / DWOS_MEM_DEVICE; device pointers must be on the
 *    context's device).  The library copies every input it keeps (geometry,
 *    data, parameters); the caller keeps ownership of all its buffers.  A
 *    call's own device inputs (query points, targets, weights) are read in
 *    place by its work on the context's stream: keep them valid and unchanged
 *    until that work has run, as for any stream-ordered CUDA call.
 *  - Work is enqueued on the context's stream (dwos_set_stream).  A call whose
 *    outputs are host memory synchronises that stream before it returns; a
 *    call whose outputs are device memory returns as soon as the work is
 *    enqueued, and a device-side failure is reported by the next dwos_sync().
 *  - Float inputs are FP32; estimator sums and all reduced outputs are FP64.
 *  - Parameter Jacobians are row-major [vertex][coordinate][parameter].
 *  - A context is not thread safe; use one context per host thread.
 */
#ifndef DWOS_H
#define DWOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dwos_ctx dwos_ctx;
typedef struct dwos_mlp dwos_mlp;       /* the control-variate network (below) */

typedef enum {
    DWOS_OK = 0,
    DWOS_ERR_INVALID_ARG = 1,     /* bad size, pointer, option or geometry */
    DWOS_ERR_CUDA = 2,            /* a CUDA runtime call failed */
    DWOS_ERR_OOM = 3,             /* device allocation failed */
    DWOS_ERR_STEP_LIMIT = 4,      /* a traversal exceeded its iteration bound */
    DWOS_ERR_TIMEOUT = 5,         /* a bounded device wait ran out (the kernel gave up instead of hanging) */
    DWOS_ERR_NOT_IMPLEMENTED = 6,
    DWOS_ERR_STATE = 7,           /* call order: e.g. eval before set_boundary */
    DWOS_ERR_OUTSIDE = 8          /* a query point lies outside Omega */
} dwos_status;

enum { DWOS_MEM_HOST = 0, DWOS_MEM_DEVICE = 1 };

/* Termination kinds stored in walk traces. */
enum { DWOS_KIND_SHELL = 0, DWOS_KIND_ROULETTE = 1, DWOS_KIND_CAPPED = 2 };

typedef struct {
    float eps;          /* shell width: a walk stops when d(x) < eps (Algorithm 1) */
    float h;            /* normal-derivative offset, Eq. (dudn_fd_estimate); h > eps */
    int K;              /* nested forward walks per differential walk (>= 1) */
    int B;              /* U-statistic batch size, Sec. 4.3 (2, 4, 8, 16 or 32) */
    int max_steps;      /* distance queries per walk phase; the last one ends the
                           phase as if the walk were in the shell (kind CAPPED) */
    uint64_t seed;      /* Philox4x32-10 key */
    int check_inside;   /* 1: reject query points outside Omega (ray parity) */
    int block_size;     /* walk-kernel threads per block; 0 = library default */
    int blocks_per_sm;  /* resident walk blocks per SM; 0 = occupancy maximum */
    int traversal;      /* distance-query search order: 0 = binary tree from the root,
                           one query per lane, bounded by the previous step's
                           element; 1 = climbing from that element's leaf with
                           the Morton-cell stop test; 2 = the 32-wide tree
                           searched by a whole warp, one query at a time;
                           3 = routed: after the seed and the outsized elements,
                           a query whose bound excludes both child boxes of the
                           binary root needs no tree search; the others are
                           searched as in order 2 (for segments, as in order 0
                           when more than 16 lanes of a warp need one at once);
                           -1 = automatic (3; with a Neumann part, 0 while the
                           Dirichlet part has fewer than 128 elements; orders 2
                           and 3 fall back to 0 without a 32-wide tree) */
    int dudn_estimator; /* du/dn at a shell hit from the K nested walks: 0 = backward
                           difference (g(xbar) - mean u(xbar - h n)) / h, Eq.
                           (dudn_fd_estimate); 1 = ball gradient at x_off = xbar - h n:
                           each nested walk first moves to y uniform on the sphere of
                           radius R = d(x_off) (no source, no roulette) and
                           contributes F(R) (n_y . n) u(y), Eq. (dudn_mc_estimate) with
                           F = d / R for sigma = 0, k / I1(kR) (2D) and k / i1(kR)
                           (3D, spherical) for k = sqrt(sigma) > 0 */
} dwos_options;

/* Per-walk record of a differential walk (32 bytes).  For a walk that reaches
 * the shell at element e with vertex weights w_i (i over the element's dim
 * vertices, w_0 = 1 - b1 [- b2]), the forward-mode derivative is
 *     udot_j = sum_i w_i ( c . J[v_i][:, j] + dg[v_i][j] )
 * where c = (dg/dn - du/dn) n - grad_Gamma(g): Eq. (wos_deriv), shell case,
 * with V_n = n . sum_i w_i J[v_i] and the boundary-data derivative of
 * Eq. (boundary_deriv_restricted) (field data) or Eq. (boundary_deriv_mapped)
 * (per-vertex data).  A walk ended by Russian roulette has elem = -1 and c = 0
 * (Algorithm 2 returns 0). */
typedef struct {
    float u;            /* u estimate of the same path (Sec. 4.1, observation 2) */
    int32_t elem;       /* terminal element (input numbering) or -1 */
    float b1, b2;       /* barycentric weights of the element's vertices 1 and 2 */
    float c[3];         /* see above; c[2] = 0 in 2D */
    uint32_t meta;      /* bits 0-23: distance queries of the main walk;
                           bits 24-25: its termination kind */
} dwos_record;

/* Optional per-walk diagnostics of a differential walk (48 bytes).  With a
 * nested control-variate table (q, t) at the main walk's element e,
 * u_off = u_plain - q disp_n - disp_t; without one u_off = u_plain. */
typedef struct {
    float dudn;         /* (g(xbar) - u_off) / h */
    float n[3];         /* oriented normal at xbar */
    float u_off;        /* mean of the K nested estimates at x_off = xbar - h n (corrected) */
    float xbar[3];      /* closest boundary point where the main walk stopped */
    float u_plain;      /* mean of the K nested estimates, uncorrected */
    float disp_n;       /* mean over the nested walks of n . (x_end - x_off) */
    float disp_t;       /* mean over the nested walks of t . (x_end - x_off) (0 without a table) */
    int32_t elem;       /* the main walk's terminal element, -1 if none */
} dwos_walk_debug;

typedef struct {
    uint64_t steps_main;    /* distance queries of main (differential/forward) walks */
    uint64_t steps_nested;  /* distance queries of nested forward walks */
    uint64_t walks;         /* main walks run */
    uint64_t capped;        /* walk phases that hit max_steps */
    uint64_t nodes_visited; /* binary BVH node fetches made by the distance queries */
    uint64_t prims_tested;  /* element distance tests made by the distance queries */
    uint64_t launches;      /* kernels this context has launched since creation */
    float kernel_ms;        /* device time of the last walk kernel (0 if unknown) */
    int blocks;             /* thread blocks of the last walk kernel */
    uint64_t wide_nodes_visited; /* 32-wide node visits (search orders 2 and 3) */
} dwos_run_stats;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device` (its own default stream until
 * dwos_set_stream).  *out receives NULL on failure. */
dwos_status dwos_create(dwos_ctx** out, int device);
/* Release every device buffer the context owns.  NULL is ignored. */
void dwos_destroy(dwos_ctx* ctx);
/* Enqueue all further work on `stream` (a cudaStream_t; NULL = legacy default). */
dwos_status dwos_set_stream(dwos_ctx* ctx, void* stream);
/* Message of the last failed call on this context ("" if none); valid until
 * the next call.  ctx may be NULL for failures of dwos_create. */
const char* dwos_last_error(const dwos_ctx* ctx);
/* Block until the context's stream is idle and report any device-side error
 * raised by earlier asynchronous calls (step-limit or outside-Omega flags). */
dwos_status dwos_sync(dwos_ctx* ctx);

/* Fill *opt with the defaults: eps 1e-3, h 1e-2, K 1, B 8, max_steps 16384,
 * seed 0x12964, check_inside 1, automatic launch shape, traversal -1 (automatic),
 * dudn_estimator 0. */
void dwos_default_options(dwos_options* opt);
/* Validate and store options (eps > 0, h > 0, K >= 1, B in {2,4,8,16,32},
 * 1 <= max_steps < 2^24). */
dwos_status dwos_set_options(dwos_ctx* ctx, const dwos_options* opt);

/* ---- problem ------------------------------------------------------------ */

/* Load the boundary (Sec. 3.1.2, explicit surface): dim 2 (segments, elem has
 * 2 ids per row) or dim 3 (triangles, 3 ids per row).  vert_ref is the
 * reference vertex array (n_vert x dim); vert_jac (n_vert x dim x n_param,
 * or NULL with n_param = 0) gives dv/dtheta, so that v(theta) = vert_ref +
 * vert_jac theta.  Builds the BVH on the device.  Resets Dirichlet data to
 * mapped g = 0 and theta to 0. */
dwos_status dwos_set_boundary(dwos_ctx* ctx, int dim, int n_vert, const float* vert_ref,
                              int n_elem, const int32_t* elem, int n_param,
                              const float* vert_jac, int mem);
/* Set theta (n_param values): v = vert_ref + vert_jac theta on the device,
 * then update the BVH for the moved vertices.  The update refits the tree's
 * boxes over its existing topology, on the device, with no host
 * synchronisation; every 64th update, and every update while search order 1
 * is selected (its Morton cells need a fresh tree), rebuilds it instead.  The
 * searches are exact over either tree, so the walks do not depend on which
 * was done, up to the choice between equally distant elements. */
dwos_status dwos_set_params(dwos_ctx* ctx, const float* theta, int mem);
/* Mapped (per-vertex, linearly interpolated) Dirichlet data, Sec. 4.1
 * "Mapped boundary data": g_vert (n_vert) and optionally dg_vert
 * (n_vert x n_param, dg_v/dtheta; NULL = 0).  dg/dn is taken as 0 (the data
 * is extended constant along the normal). */
dwos_status dwos_set_dirichlet_mapped(dwos_ctx* ctx, const float* g_vert, const float* dg_vert,
                                      int mem);
/* Restricted Dirichlet data, Sec. 4.1 "Restricted boundary data": the field
 * g(x) = c0 + c.x + x^T A x, independent of theta; coeffs (host, 10 values)
 * = {c0, c_x, c_y, c_z, A_xx, A_yy, A_zz, A_xy, A_xz, A_yz}. */
dwos_status dwos_set_dirichlet_field(dwos_ctx* ctx, const double* coeffs);
/* Screening sigma >= 0 and constant source f (of -Lap u + sigma u = f). */
dwos_status dwos_set_pde(dwos_ctx* ctx, float sigma, float f);
/* Mixed Dirichlet / Neumann boundary (Sec. 3.4, Eq. mixed_bvp with Robin
 * coefficient 0: a reflecting boundary, as in the paper's thermal design,
 * Sec. 6.3, until dwos_set_neumann_data gives it data du/dn).  flags (n_elem int32, host or device by
 * mem): 1 marks an element of the Neumann part, 0 of the Dirichlet part; NULL
 * or all zeros makes every element Dirichlet again.  The Dirichlet part must
 * not be empty.  With a Neumann part every walk-running call (dwos_eval,
 * dwos_vjp, dwos_grad_l2, dwos_grad_l2_product, dwos_walk_records) runs walks
 * on stars (Sawhney et al. 2023): from x the walk takes the star-shaped
 * region of the ball of radius R = max(min(distance to the Dirichlet part
 * - c, distance to the closest Neumann silhouette point), eps - c), with the
 * clearance c = 1e-3 eps, that x sees without crossing the Neumann part,
 * moves along a uniform direction (into the domain's half-space when x lies
 * on the Neumann part, into the wedge of the two sides at an edge) to the
 * first Neumann
 * crossing or the sphere, survives Russian roulette with probability
 * |S| t^(d-1) |G_R'(t)| for the step length t, and counts a source sample of
 * the ball where x sees it; walks end in the eps-shell of the Dirichlet part
 * only.  The differential walk nests there (Sec. 4.2, Eq. mixed_bvp_deriv):
 * the Neumann part contributes no boundary term, and its vertices' motion
 * (for instance the tangential stretch of a side next to a moving Dirichlet
 * part) enters only through the geometry.  Query points lie in the interior
 * or on the Neumann part (the thermal design observes its temperature there):
 * a point within 1e-3 eps of the Neumann part starts its walk on the closest
 * Neumann element (at a vertex shared by two, the search's pick), with that
 * element's normal oriented out of the domain (the point 1e-3 of the
 * element's size behind its centre is inside); such points count as inside.
 * Records number elements as the input does.  Not available with
 * a Neumann part: the ball-gradient du/dn estimator, control variates,
 * batches, dwos_eval_static and the shape-functional calls
 * (DWOS_ERR_NOT_IMPLEMENTED / DWOS_ERR_INVALID_ARG).  dwos_closest_point
 * then answers for the Dirichlet part, dwos_inside for the whole boundary.
 * A silhouette point lies where the Neumann part ends or turns: where it runs
 * straight on through a vertex (flat across an edge: unit directions or
 * normals within a relative 1e-6) it has none.  Builds a BVH for each part
 * and one over the silhouette candidates (every vertex / edge where the part
 * ends or turns, and every one with a vertex whose Jacobian row is nonzero);
 * dwos_set_params updates all three.  Synchronises. */
dwos_status dwos_set_neumann(dwos_ctx* ctx, const int32_t* flags, int mem);
/* Neumann data on the Neumann part (Sec. 3.4, Eq. mixed_bvp with Robin
 * coefficient 0 and data h = du/dn, n the normal out of the domain):
 * h (n_elem floats, host or device by mem, constant on each element, read on
 * the Neumann elements only; NULL or all zeros: a reflecting boundary again).
 * Each walk-on-stars step then adds one sample of (1 / a(x)) times the
 * integral of G_R(x, z) h(z) over the Neumann boundary in its ball that x
 * sees (Green's second identity on the star), a(x) the share of directions
 * into the domain at x (1 inside, 1/2 on a side, (pi - the angle between the
 * two normals) / 2 pi at an edge): a Neumann element within R (1 - 1e-4) of x
 * (an element that only touches the ball at a silhouette point is left out,
 * and so is one wholly behind a side the walk sits on: every vertex more than
 * 2e-4 eps behind the side's plane), drawn with probability proportional to its
 * length (area) among them by per-element keys, and a uniform
 * point z on it; the sample is A G_R(|z - x|) h / a(x) when |z - x| < R and x
 * sees z (A the total measure of those elements), else 0.  The data does not
 * depend on theta, so it enters du/dtheta only through the nested walks at
 * the Dirichlet shell (Sec. 4.2, Eq. mixed_bvp_deriv).  Kept across
 * dwos_set_neumann and dwos_set_params; dwos_set_boundary clears it.  Values
 * must be finite (DWOS_ERR_INVALID_ARG).  Synchronises. */
dwos_status dwos_set_neumann_data(dwos_ctx* ctx, const float* h, int mem);

/* Bound on the BVH node fetches (binary nodes, or 32-wide node visits) that one
 * distance query of a walk may make; 0 (the default) keeps the trees' own
 * bounds, which a valid tree never reaches.  A query that exceeds the bound
 * keeps the closest element it has found, its walk continues, and the call
 * reports DWOS_ERR_STEP_LIMIT (at once for host outputs, else at dwos_sync).
 * It exists to exercise that failure path without a fault.  max_fetches >= 0. */
dwos_status dwos_set_traversal_budget(dwos_ctx* ctx, int max_fetches);

/* ---- estimators --------------------------------------------------------- */

/* Forward estimates at n_query points (xq: n_query x dim), walks_per_point
 * walks each.  u_mean, u_se: n_query FP64 (mean and standard error).  If
 * du_mean is not NULL, runs differential walks (Algorithm 2) and also returns
 * the forward-mode derivative du_mean (n_query x n_param) and, if not NULL,
 * its standard error du_se.  Walk w of point p uses Philox walk id
 * p * walks_per_point + w. */
dwos_status dwos_eval(dwos_ctx* ctx, int n_query, const float* xq, int walks_per_point,
                      double* u_mean, double* u_se, double* du_mean, double* du_se, int mem);

/* Reverse mode with a caller-supplied cotangent w (n_query): grad_param
 * (n_param) = sum_p w_p E[udot_p], and grad_vert (n_vert x dim, or NULL) the
 * same product with respect to the vertex positions.  Draws its own walks
 * (ids start at walk_id_base), independent of any earlier call that produced
 * w when the bases differ. */
dwos_status dwos_vjp(dwos_ctx* ctx, int n_query, const float* xq, const float* w,
                     int walks_per_point, uint64_t walk_id_base, double* grad_param,
                     double* grad_vert, int mem);

/* Squared loss L = 1/2 sum_p (u_p - uref_p)^2 (Eq. functional with a
 * point mask; Eq. squared_loss_deriv) and its gradient with the U-statistic
 * product estimator in batches of B consecutive walks (Eq. ustatistics;
 * walks_per_point must be a multiple of B).  loss (1 value), grad_param
 * (n_param) and grad_vert (n_vert x dim, may be NULL). */
dwos_status dwos_grad_l2(dwos_ctx* ctx, int n_query, const float* xq, const float* uref,
                         int walks_per_point, uint64_t walk_id_base, double* loss,
                         double* grad_param, double* grad_vert, int mem);

/* The same squared-loss gradient with a choice of product estimator for
 * u udot (Sec. 4.3): product 0 = U-statistic (as dwos_grad_l2), 1 =
 * correlated (Eq. correlated_product: mean u and mean udot of all W walks;
 * biased), 2 = uncorrelated (Eq. uncorrelated_product: u from walks
 * 0 .. W/2 - 1 of each point, udot from the others; W even).  The loss is
 * always that of the mean of all W walks. */
dwos_status dwos_grad_l2_product(dwos_ctx* ctx, int n_query, const float* xq, const float* uref,
                                 int walks_per_point, uint64_t walk_id_base, int product, double* loss,
                                 double* grad_param, double* grad_vert, int mem);

/* dwos_grad_l2 with a control variate and training samples (device pointers
 * only).  cv_grad (n_query x dim, or NULL) is the spatial gradient of a smooth
 * surrogate of u at the query points (e.g. the learned network's,
 * dwos_mlp_eval).  Each sphere step of a walk moves it by d w with w uniform on
 * the sphere and independent of whether the step happens (shell test and
 * roulette use other draws), so g . (d w) has mean zero for any fixed g.  A
 * walk from x0 therefore contributes u - cv_grad(x0) . (x1 - x0), with x1 its
 * point after the first step (cv_whole_walk = 0), or u - cv_grad(x0) .
 * (x_end - x0), with x_end where its main walk stopped (cv_whole_walk = 1, the
 * sum of all its steps).  cv_elem (n_elem x 4 floats, 16-byte aligned, or
 * NULL) holds per boundary element a surrogate of grad u there, split as
 * (q, t0, t1, t2): grad u ~ q n + t with n the walk's oriented normal at the
 * hit (q stands for du/dn, t for the tangential gradient of the data).  Each
 * nested walk launched from x_off = xbar - h n at a shell hit on element e
 * then contributes u - (q n + t) . (x_end - x_off) to the backward difference
 * of Eq. (dudn_fd_estimate), again a zero-mean correction.
 * Either way the loss gradient stays unbiased for any surrogate (Sec. 4.3's
 * U-statistic weights use the corrected u).  samples (4 floats per
 * walk, or NULL): (x1, estimate of u at x1) for walks that moved, NaN x
 * otherwise.  debug (or NULL): per-walk diagnostics (xbar, du/dn).  u_se_pair (2 x
 * n_query, or NULL): per-point standard errors of u without and with the
 * control variate.  Asynchronous. */
dwos_status dwos_grad_l2_cv(dwos_ctx* ctx, int n_query, const float* xq, const float* uref, int walks_per_point,
                            uint64_t walk_id_base, const float* cv_grad, int cv_whole_walk, const float* cv_elem,
                            float* samples, dwos_walk_debug* debug, double* loss, double* grad_param,
                            double* u_se_pair);

/* The nested walks' control-variate table for dwos_grad_l2_cv (2D boundaries):
 * table (device, n_elem x 4 floats, 16-byte aligned) receives per element
 * (q, t0, t1, 0) with q the network's du/dn head (output 1) at the element's
 * centre and t the tangential gradient of the Dirichlet data on the element
 * ((g1 - g0) / |d|^2 d for vertex data, grad g minus its normal part at the
 * centre for field data), all at the current vertices.  Runs on the context's
 * stream (the network's stream is set to it).  Asynchronous. */
dwos_status dwos_cv_table(dwos_ctx* ctx, dwos_mlp* mlp, float* table);

/* Training rows for the control-variate network (dwos_mlp_train_step) from
 * one dwos_grad_l2_cv call's per-walk outputs, all device memory: samples
 * (n_walks x 4 floats, the call's `samples`) and debug (n_walks records, or
 * NULL).  The walks offset, offset + stride, ... are used (R = ceil((n_walks -
 * offset) / stride) of them).  Rows 0 .. R-1 train output 0 (u) at the main
 * walk's first-step point x1 on its estimate of u there (mask 0 where the walk
 * never moved).  With debug, rows R .. 2R-1 train output 1 (du/dn) at the hit
 * point xbar on r / disp_n with r = u_plain - g(xbar) - disp_t and g(xbar) =
 * u_off + h du/dn (h the context's offset option): the weighted least-squares
 * fit, weight |disp_n|, of the slope that minimises the variance of the nested
 * walks' corrected mean, the weights scaled by sqrt(q_weight / mean r^2) over
 * the hit walks so that both heads' losses have comparable size; rows of walks
 * that did not reach the shell have mask 0.  x, target and mask receive
 * 2 x (rows) floats each (room for 2R rows); *n_rows (host) the row count.
 * Asynchronous on the context's stream. */
dwos_status dwos_cv_training_set(dwos_ctx* ctx, long long n_walks, const float* samples, const dwos_walk_debug* debug,
                                 long long stride, long long offset, float q_weight, float* x, float* target,
                                 float* mask, long long* n_rows);

/* Measurement helper (not part of the method): read bandwidth of an
 * L2-resident buffer of `bytes` bytes on `device`, read `reps` times by a
 * coalesced grid-stride kernel; the roof against which the walk kernel's
 * tree traffic (which stays on chip) is compared.  Synchronous. */
dwos_status dwos_probe_l2_read(int device, size_t bytes, int reps, double* gbs);

/* ---- volume-integrated shape functional ----------------------------------
 * J(theta) = int_Omega M(x) 1/2 (u(x) - uref(x))^2 dx (Eq. functional, M the
 * indicator of an axis-aligned box) and its derivative, Eq. functional_deriv:
 *   dJ/dtheta = int_Omega M (u - uref) udot dx + int_Gamma M V_n 1/2 (u - uref)^2 dA.
 * The domain term: dwos_sample_domain draws n_try points uniformly in the
 * box (Philox4x32-10, key = seed, counter = (i, 0, 0, 0xD0A1), words 0..dim-1
 * mapped as for the walks), keeps those inside Omega (ray parity), in
 * candidate order, in points (device, n_try x dim floats of room), and
 * returns their number and the weight |box| / n_try each carries (an
 * unbiased quadrature of the box integral); dwos_grad_l2_weighted is
 * dwos_grad_l2 with those weights per point (loss = sum_p w_p 1/2 (u_p -
 * uref_p)^2, the U-statistic product per point scaled by w_p).  The boundary
 * term: dwos_boundary_term_l2 integrates M V_n 1/2 (g - uref)^2 over the
 * boundary (u = g there), with mapped vertex data g and uref_vert (n_vert
 * values, or NULL for 0) both linear on each element, M the box indicator at
 * the element's centre, and V_n along the outward normal (oriented by the
 * inside test of a point just behind the element); the per-element integrals
 * are exact.  grad_param receives n_param values (host or device by mem).
 * Both calls synchronise. */
dwos_status dwos_sample_domain(dwos_ctx* ctx, int n_try, const float* box_lo, const float* box_hi, uint64_t seed,
                               float* points, int* n_inside, float* weight);
dwos_status dwos_grad_l2_weighted(dwos_ctx* ctx, int n_query, const float* xq, const float* uref,
                                  const float* point_weight, int walks_per_point, uint64_t walk_id_base,
                                  double* loss, double* grad_param, double* grad_vert, int mem);
dwos_status dwos_boundary_term_l2(dwos_ctx* ctx, const float* box_lo, const float* box_hi, const float* uref_vert,
                                  double* grad_param, int mem);

/* ---- boundary loss of the general shape functional ------------------------
 * App. C, Eq. general_functional: J_b(theta) = int_Gamma m(y) l_b(u(y)) dA
 * with l_b(u) = 1/2 (u - ub)^2, m the indicator of an axis-aligned box (taken
 * at each element's centre and held fixed) and ub_vert the target per vertex
 * (n_vert values, host or device by mem, or NULL for 0).  On a Dirichlet
 * boundary u = g, and the du/dn terms of Eq. general_functional_deriv cancel
 * against udot = gdot - V_n du/dn (Eq. bvp_deriv), so no walk is needed: the
 * call returns J_b and its exact derivative for mapped vertex data g, linear
 * on each element, through the element measures (the discrete mean-curvature
 * term; vertices move by the Jacobian given to dwos_set_boundary) and through
 * dg/dtheta (dwos_set_dirichlet_mapped).  loss receives 1 value and
 * grad_param n_param values (host or device by mem).  Field data:
 * DWOS_ERR_NOT_IMPLEMENTED.  Synchronises.  With dwos_sample_domain,
 * dwos_grad_l2_weighted and dwos_boundary_term_l2 this gives the derivative
 * of the whole general functional. */
dwos_status dwos_boundary_loss_l2(dwos_ctx* ctx, const float* box_lo, const float* box_hi, const float* ub_vert,
                                  double* loss, double* grad_param, int mem);

/* The current vertex positions (n_vert x dim floats: reference + J theta),
 * host or device by mem.  Synchronises for host memory. */
dwos_status dwos_get_vertices(const dwos_ctx* ctx, float* vert, int mem);

/* Sizes of the acceleration structures built by dwos_set_boundary /
 * dwos_set_params: info[0..5] = elements, elements in the binary tree,
 * outsized elements kept out of it, binary inner nodes, 32-wide nodes, levels
 * of the 32-wide tree.  Synchronous (host array). */
dwos_status dwos_bvh_info(const dwos_ctx* ctx, int32_t* info);

/* Raw per-walk records (n_query x walks_per_point rows, row p*W + w, Philox
 * walk id walk_id_base + p*W + w).  differential = 0 runs Algorithm 1 only
 * (record.u, record.elem, record.b*, meta; c = 0).  trace (optional,
 * (K+1) words per walk: bits 0-29 distance queries of that phase, bits 30-31
 * its termination kind; nested slots of walks that never reached the shell
 * are 0xFFFFFFFF) and debug (optional) are written when not NULL. */
dwos_status dwos_walk_records(dwos_ctx* ctx, int n_query, const float* xq, int walks_per_point,
                              uint64_t walk_id_base, int differential, dwos_record* records,
                              uint32_t* trace, dwos_walk_debug* debug, int mem);

/* Statistics of the last walk launch on this context (synchronises). */
dwos_status dwos_last_stats(dwos_ctx* ctx, dwos_run_stats* out);

/* ---- geometry queries and primitives (used by tests and tools) ---------- */

/* DistanceToBoundary (Algorithm 1) through the BVH for n points: dist (n),
 * elem (n, input numbering), bary (n x 2, weights of vertices 1 and 2). */
dwos_status dwos_closest_point(dwos_ctx* ctx, int n, const float* p, float* dist, int32_t* elem,
                               float* bary, int mem);
/* The same query seeded, as a walk step is, with a known element: hint_elem
 * (n, input numbering; -1 = no hint) bounds the distance before the search,
 * which then climbs the BVH from that element's leaf.  Results equal
 * dwos_closest_point's for any hints (the hint only changes the work done). */
dwos_status dwos_closest_point_hint(dwos_ctx* ctx, int n, const float* p, const int32_t* hint_elem, float* dist,
                                    int32_t* elem, float* bary, int mem);
/* 1 if the point lies inside the region the boundary encloses (odd number of
 * ray crossings), else 0. */
dwos_status dwos_inside(dwos_ctx* ctx, int n, const float* p, int32_t* inside, int mem);
/* Philox4x32-10 (Salmon et al., SC'11) on the device: out[4i..4i+3] =
 * Philox(ctr[4i..4i+3], key[0..1]) for i < n.  ctx selects the device. */
dwos_status dwos_philox4x32_10(dwos_ctx* ctx, int n, const uint32_t* ctr, const uint32_t* key,
                               uint32_t* out, int mem);
/* The two ball weights of a walk step (Sec. 3.3.1, Algorithm 1), evaluated on
 * the device exactly as the walk kernel does, for n pairs (d[i], u[i]) with
 * d > 0 the ball radius and u in (0, 1) the uniform that places the source
 * sample at r = d u^(1/dim): source[i] = |B(d)| G_d(r), the source estimate
 * per unit f, and alpha[i] = P(d) |dB(d)|, the Russian-roulette survival
 * probability; G and P are the screened Green's function and Poisson kernel
 * of the ball for k = sqrt(sigma) (2D: G = (K0(kr) - K0(kd) I0(kr)/I0(kd)) /
 * 2 pi, alpha = 1 / I0(kd); 3D: G = sinh(k(d - r)) / (4 pi r sinh kd),
 * alpha = kd / sinh kd; the Laplace limits at sigma = 0).  Either output may
 * be NULL.  Inputs and outputs are host or device memory by mem; sizes n. */
dwos_status dwos_ball_weights(dwos_ctx* ctx, int dim, float sigma, int n, const float* d, const float* u,
                              float* source, float* alpha, int mem);
/* The modified Bessel functions K0(x) and K1(x), x > 0, as the 2D source
 * weight and the walk-on-stars step weight evaluate them (the polynomial
 * approximations 9.8.5-9.8.8 of Abramowitz & Stegun in FP32): out[i] =
 * K0(x[i]) or K1(x[i]) for i < n, host or device memory by mem. */
dwos_status dwos_bessel_k0(dwos_ctx* ctx, int n, const float* x, float* out, int mem);
dwos_status dwos_bessel_k1(dwos_ctx* ctx, int n, const float* x, float* out, int mem);
/* The walk-on-stars step's survival weight |S^(d-1)| t^(d-1) |G_R'(t)| for
 * n pairs (t[i], R[i]), 0 < t <= R, evaluated as the walk kernel does
 * (see dwos_set_neumann). */
dwos_status dwos_star_weight(dwos_ctx* ctx, int dim, float sigma, int n, const float* t, const float* R, float* out,
                             int mem);

/* ---- batched problems ----------------------------------------------------
 * Many independent reverse-mode problems in one pass: each job is a
 * dwos_grad_l2 (Sec. 4.3, U-statistic squared-loss gradient) on its own
 * context (boundary, BVH, data, PDE and options of that context).  The jobs of
 * one dimension share a persistent walk launch over a table of up to 64
 * problem descriptors, so the tail of long walks is paid once per launch.  A
 * pass enqueues only kernels and memsets on the batch's stream and can be
 * captured into a CUDA graph.  Contexts must outlive the batch and must not be
 * changed (boundary, parameters, data, options) while it is used; create a new
 * batch after such changes.  All pointers in a job are device memory on the
 * contexts' device, owned by the caller. */
typedef struct dwos_batch dwos_batch;
typedef struct {
    dwos_ctx* ctx;          /* the problem */
    int n_query;            /* >= 1 */
    const float* xq;        /* n_query x dim query points */
    int walks_per_point;    /* multiple of the context's B */
    const float* uref;      /* n_query targets of the squared loss */
    uint64_t walk_id_base;  /* Philox walk id of the job's first walk */
    double* loss;           /* 1 value */
    double* grad_param;     /* n_param values (may be NULL if n_param = 0) */
    double* u_mean;         /* n_query values or NULL */
} dwos_batch_job;

/* Validate the jobs, run the inside test once (DWOS_ERR_OUTSIDE if a point is
 * outside its domain), allocate every buffer a pass needs and build the
 * descriptor tables.  stream: cudaStream_t of all passes (a non-default stream
 * is needed for graph capture).  Synchronises. */
dwos_status dwos_batch_create(dwos_batch** out, const dwos_batch_job* jobs, int n_jobs, void* stream);
void dwos_batch_destroy(dwos_batch* b);
const char* dwos_batch_last_error(const dwos_batch* b);
/* Enqueue one pass: walks of every job, then each job's scatter, GEMV, mean
 * and loss.  Asynchronous; allocates nothing; capturable. */
dwos_status dwos_batch_run(dwos_batch* b);
/* Capture one pass into a CUDA graph (replaces an earlier one). */
dwos_status dwos_batch_capture(dwos_batch* b);
/* Replay the captured graph on the batch's stream. */
dwos_status dwos_batch_launch(dwos_batch* b);
/* Time the walk launch of each dimension group over block size (128, 256),
 * resident blocks per SM (1, 2, 4, ... up to the occupancy limit) and the
 * distance-query search order (dwos_options.traversal 0 to 3), reps passes
 * each, and keep the fastest; recaptures the graph if one exists.
 * Synchronises. */
dwos_status dwos_batch_autotune(dwos_batch* b, int reps);
/* The configuration in use for dimension dim and, after autotuning, its walk time. */
dwos_status dwos_batch_config(const dwos_batch* b, int dim, int* block_size, int* blocks_per_sm, int* traversal,
                              float* walk_ms);
/* Walk statistics of the last pass (summed over launches; synchronises). */
dwos_status dwos_batch_stats(dwos_batch* b, dwos_run_stats* out);
/* enable = 1: later passes also write each walk's trace ((K + 1) words per
 * walk, the layout of dwos_walk_records); 0: stop.  Allocates (or frees) the
 * trace buffer and recaptures the graph if one exists.  Synchronises. */
dwos_status dwos_batch_trace(dwos_batch* b, int enable);
/* The per-walk records of job `job` from the last pass (n_query x
 * walks_per_point rows, row p*W + w, Philox walk id walk_id_base + p*W + w,
 * layout of dwos_record) and, if trace is not NULL, its traces (traces must be
 * on).  Host or device memory by mem.  Synchronises the batch's stream. */
dwos_status dwos_batch_records(dwos_batch* b, int job, dwos_record* records, uint32_t* trace, int mem);

/* ---- learned control variate ---------------------------------------------
 * The paper points to variance reduction for WoS (Sec. 2, Sec. 7) without
 * fixing one; this network is the learned control variate of the 2D
 * shape-from-diffusion workload.  Features (x, y, sin pi x, sin pi y,
 * sin pi (x + y)) -> four tanh layers of 64 -> 8 linear outputs, of which
 * output 0 estimates u and output 1 du/dn.  Training and evaluation run on
 * the tensor cores (tcgen05, accumulators in TMEM): every matrix-product input
 * (weights, activations, deltas) is BF16, sums are FP32, biases, tanh and the
 * loss FP32, and tanh' = 1 - a^2 uses the activation as stored (BF16);
 * parameters are FP32 with Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * Flat parameter layout: W1 (64 x 16), b1 (64), W2 (64 x 64), b2, W3, b3, W4,
 * b4, W5 (8 x 64), b5 (8), W[out][in] row-major.  Loss: (1/n) sum_s sum_k
 * mask[s][k] (out[s][k] - target[s][k])^2 over k in {0, 1}.  Points x,
 * targets and masks are n x 2 row-major; `mem` applies to every pointer. */
#define DWOS_MLP_NPARAM 14088
dwos_status dwos_mlp_create(dwos_mlp** out, int device);   /* parameters zero */
void dwos_mlp_destroy(dwos_mlp* mlp);
const char* dwos_mlp_last_error(const dwos_mlp* mlp);
dwos_status dwos_mlp_set_stream(dwos_mlp* mlp, void* stream);
/* Load parameters (DWOS_MLP_NPARAM floats) and reset the Adam state. */
dwos_status dwos_mlp_set_params(dwos_mlp* mlp, const float* params, int mem);
dwos_status dwos_mlp_get_params(dwos_mlp* mlp, float* params, int mem);
/* Loss and gradient (DWOS_MLP_NPARAM floats) on n samples, no update. */
dwos_status dwos_mlp_loss_grad(dwos_mlp* mlp, int n, const float* x, const float* target, const float* mask,
                               float* grad, double* loss, int mem);
/* One Adam step with learning rate lr on n samples; loss (may be NULL) is the
 * loss before the step. */
dwos_status dwos_mlp_train_step(dwos_mlp* mlp, int n, const float* x, const float* target, const float* mask,
                                float lr, double* loss, int mem);
/* Output 0 (u), its gradient d u / d(x, y) (n x 2, the backward pass of
 * output 0 in the same arithmetic) and output 1 (du/dn) at n points; any
 * output may be NULL. */
dwos_status dwos_mlp_eval(dwos_mlp* mlp, int n, const float* x, float* u, float* grad_u, float* q, int mem);

/* Wait for the network's queued work and report a tensor-core product that did
 * not complete within its bounded wait (DWOS_ERR_TIMEOUT; the kernels give up
 * instead of hanging).  Calls with host buffers check this themselves.  The
 * failure is reported once; the next call starts clean. */
dwos_status dwos_mlp_sync(dwos_mlp* mlp);
/* The bounded-wait failure path without a fault: a kernel waits, with the
 * training kernel's bounded mbarrier wait, on a barrier that nothing arrives
 * at (no copy or product is issued), gives up after `polls` tries (1 ..
 * 2^24) and raises the network's timeout flag.  Returns DWOS_ERR_TIMEOUT, as
 * a stalled product would; the network stays usable.  Synchronises. */
dwos_status dwos_mlp_wait_probe(dwos_mlp* mlp, int polls);

/* ---- allocation-free evaluation ------------------------------------------
 * The paper has no counterpart to this entry point.  It is dwos_eval for
 * callers that cannot allocate device memory during the call: hosts whose
 * device memory belongs to another allocator (a framework's caching pool) or
 * to a fixed budget set aside at start-up, and loops that cannot afford the
 * implicit device synchronisation that cudaMalloc and cudaFree bring.
 *
 * It runs the same kernels as dwos_eval (inside test if enabled, walks with
 * walk id p * W + w, per-point reductions) but keeps all scratch in one fixed
 * array compiled into the library: about 9.4 MB on every GPU that loads the
 * library, held until the process exits.  It never calls cudaMalloc or
 * cudaFree.  Limits and rules:
 *  - n_query * walks_per_point <= DWOS_STATIC_MAX_WALKS, else
 *    DWOS_ERR_INVALID_ARG with a message saying so;
 *  - xq (n_query x dim) and every output are device pointers on the context's
 *    device (outputs as in dwos_eval; du_mean / du_se may be NULL);
 *  - the boundary, data and options must already be set on the context (those
 *    calls do allocate);
 *  - the first call on a device does a one-time set-up: it looks up the
 *    array's device address, with that device current; make that first call
 *    before any stream capture begins.  The address belongs to the device's
 *    primary context, so a cudaDeviceReset in the process invalidates it;
 *  - all calls, from every context in the process, share the one array, which
 *    keeps the previous call's contents (the counters are cleared by each
 *    call): calls whose work overlaps on the GPU race and must be ordered by
 *    the caller, e.g. by issuing them on one stream;
 *  - the work is asynchronous on the context's stream; device-side errors are
 *    not reported (the counters live in the shared array); dwos_last_stats
 *    does not describe these calls. */
#define DWOS_STATIC_MAX_WALKS 262144
dwos_status dwos_eval_static(dwos_ctx* ctx, int n_query, const float* xq, int walks_per_point,
                             double* u_mean, double* u_se, double* du_mean, double* du_se);

#ifdef __cplusplus
}
#endif
#endif /* DWOS_H */
