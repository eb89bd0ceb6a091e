/*
 * FP64 CPU oracle for Differential Walk on Spheres (Miller, Sawhney, Crane,
 * Gkioulekas, ACM TOG 43(6), 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or constant table with the
 * CUDA library: the random-number generator, the sampling formulas, the
 * Green's-function weights and the closest-point queries below are written
 * independently from their published definitions.
 *
 * Everything is double precision and deliberately naive: the closest point is
 * a brute-force minimum over every boundary element, and each walk follows the
 * steps of the paper's Algorithm 1 (WalkOnSpheres) or Algorithm 2
 * (DiffWalkOnSpheres) in the paper's order.
 *
 * Readings of the paper that this file fixes (each is also listed in the
 * design notes):
 *  - Source sign.  Eq. (bvp) in Sec. 3.2 writes  Lap u - sigma u = f, but
 *    Algorithm 1 adds +G f / p with the positive ball Green's function.  The
 *    oracle follows the algorithm: f is the source of  -Lap u + sigma u = f.
 *  - G and P on a ball are not printed (Sec. 3.3.1 defers to WoSt App. A).
 *    They are derived here from the PDE:
 *      3D: G(r) = sinh(k(R-r)) / (4 pi r sinh(kR)),      alpha = kR / sinh(kR)
 *      2D: G(r) = (K0(kr) - K0(kR) I0(kr)/I0(kR)) / 2pi,  alpha = 1 / I0(kR)
 *    with k = sqrt(sigma); sigma = 0 gives the Laplace limits and alpha = 1.
 *  - Shell test is strict, d < eps (Algorithm 1 and 2).
 *  - Russian roulette stops the walk when alpha < U (Algorithm 1 and 2); the
 *    survivor keeps weight 1.
 *  - BoundaryNormal (Algorithm 2) is the geometric normal of the closest
 *    element, oriented so that n . (xbar - x) >= 0, i.e. away from the walk.
 *  - Mapped boundary data (Eq. boundary_deriv_mapped): the reference data is
 *    extended constant along the normal, so dg/dn = 0 and the tangential term
 *    is  -grad_Gamma(g) . V  with V the interpolated vertex velocity.
 *  - A walk phase is capped at max_steps distance queries: the last allowed
 *    query treats the walk as if it had reached the shell at its current
 *    closest point (kind CAPPED).  The paper sets no cap.
 *  - Mixed Dirichlet-Neumann boundaries (Sec. 3.4, Eq. mixed_bvp, with Robin
 *    coefficient 0; zero Neumann data as in the thermal design of Sec. 6.3,
 *    or data du/dn per element, see neumann_data_sample below): the walks are
 *    walks on stars (see wost_walk below), and the differential walk nests at
 *    the Dirichlet shell only (Sec. 4.2, Eq. mixed_bvp_deriv).  The star
 *    radius is at least eps.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), keyed by
 * the seed; counter = (walk id lo, walk id hi, step, (phase << 8) | block).
 * Block 0 of a step gives the sphere direction (words 0, 1) and the roulette
 * draw (word 2); block 1 gives the ball sample for the source (words 0, 1, 2).
 * A 32-bit word x maps to the uniform ((x >> 9) * 2 + 1) * 2^-24 in (0, 1).
 */
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <utility>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double kPi = 3.14159265358979323846;

/* ---------------------------------------------------------------------------
 * Philox4x32-10, written from the SC'11 paper's definition: ten rounds of two
 * 32x32->64 multiplications, with a Weyl sequence bumping the 64-bit key.
 * ------------------------------------------------------------------------- */
void philox4x32_10(const uint32_t in_ctr[4], const uint32_t in_key[2], uint32_t out[4]) {
    const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = in_ctr[0], c1 = in_ctr[1], c2 = in_ctr[2], c3 = in_ctr[3];
    uint32_t k0 = in_key[0], k1 = in_key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = M0 * (uint64_t)c0;
        uint64_t p1 = M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double to_uniform(uint32_t x) {
    /* odd multiples of 2^-24 in (0, 1): never 0, never 1 */
    return (double)((x >> 9) * 2u + 1u) * (1.0 / 16777216.0);
}

struct Draws { double u[3]; };

Draws draw(uint32_t seed_lo, uint32_t seed_hi, uint64_t walk_id, uint32_t step,
           uint32_t phase, uint32_t block) {
    uint32_t ctr[4] = {(uint32_t)walk_id, (uint32_t)(walk_id >> 32), step, (phase << 8) | block};
    uint32_t key[2] = {seed_lo, seed_hi};
    uint32_t out[4];
    philox4x32_10(ctr, key, out);
    Draws d;
    d.u[0] = to_uniform(out[0]);
    d.u[1] = to_uniform(out[1]);
    d.u[2] = to_uniform(out[2]);
    return d;
}

}  // namespace

extern "C" {

/* Scene description (own layout; unrelated to the CUDA library's header). */
typedef struct {
    int dim;                 /* 2: line segments, 3: triangles */
    int n_vert;
    const double* vert;      /* n_vert * dim */
    int n_elem;
    const int* elem;         /* n_elem * dim vertex ids */
    int n_param;
    const double* jac;       /* n_vert * dim * n_param, [v][k][j]; NULL: no shape params */
    int data_kind;           /* 0: mapped per-vertex data, 1: restricted field */
    const double* g_vert;    /* n_vert (mapped) */
    const double* dg_vert;   /* n_vert * n_param or NULL (mapped) */
    int field_kind;          /* unused by the formulas; kept for bookkeeping */
    double field[10];        /* g = c0 + c.x + x^T A x: c0, c[3], Axx Ayy Azz Axy Axz Ayz */
    double sigma;
    double f;                /* constant source of -Lap u + sigma u = f */
    double eps;
    double h;
    int K;                   /* nested forward walks per differential walk */
    int max_steps;           /* distance queries per walk phase */
    uint32_t seed_lo;
    uint32_t seed_hi;
    const double* cv_elem;   /* per element (q, t0, t1, t2): surrogate grad u = q n + t for the nested
                                walks' control variate, or NULL */
    int dudn_mode;           /* 0: backward difference, Eq. (dudn_fd_estimate); 1: ball gradient at the
                                offset point, Eq. (dudn_mc_estimate) */
    const int* neumann;      /* n_elem flags, 1: element of the (reflecting) Neumann boundary; NULL: all
                                elements are Dirichlet */
    const double* neumann_h; /* n_elem Neumann data h = du/dn (n out of the domain), read on the Neumann
                                elements only; NULL: zero (a reflecting boundary) */
} oracle_scene;

enum { KIND_SHELL = 0, KIND_ROULETTE = 1, KIND_CAPPED = 2 };

void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
    philox4x32_10(ctr, key, out);
}

double oracle_uniform(uint32_t x) { return to_uniform(x); }

/* ---------------------------------------------------------------------------
 * Closest point on one element.
 * Segment: project onto the line, clamp the parameter to [0, 1].
 * Triangle: the Voronoi-region case analysis of Ericson, Real-Time Collision
 * Detection, Sec. 5.1.5 (vertex regions, edge regions, face region).
 * Returns the squared distance; bary receives the weights of v1 (and v2).
 * ------------------------------------------------------------------------- */
static double closest_on_segment(const double* p, const double* a, const double* b,
                                 double* xbar, double* bary) {
    double ab[2] = {b[0] - a[0], b[1] - a[1]};
    double ap[2] = {p[0] - a[0], p[1] - a[1]};
    double len2 = ab[0] * ab[0] + ab[1] * ab[1];
    double t = len2 > 0 ? (ap[0] * ab[0] + ap[1] * ab[1]) / len2 : 0.0;
    if (t < 0) t = 0;
    if (t > 1) t = 1;
    xbar[0] = a[0] + t * ab[0];
    xbar[1] = a[1] + t * ab[1];
    bary[0] = t;
    bary[1] = 0;
    double dx = p[0] - xbar[0], dy = p[1] - xbar[1];
    return dx * dx + dy * dy;
}

static inline double dot3(const double* u, const double* v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; }

static double closest_on_triangle(const double* p, const double* a, const double* b, const double* c,
                                  double* xbar, double* bary) {
    double ab[3], ac[3], ap[3];
    for (int i = 0; i < 3; ++i) { ab[i] = b[i] - a[i]; ac[i] = c[i] - a[i]; ap[i] = p[i] - a[i]; }
    double w1 = 0, w2 = 0;  /* weights of b and c */
    double d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    if (d1 <= 0 && d2 <= 0) {                       /* vertex region a */
        w1 = 0; w2 = 0;
    } else {
        double bp[3];
        for (int i = 0; i < 3; ++i) bp[i] = p[i] - b[i];
        double d3 = dot3(ab, bp), d4 = dot3(ac, bp);
        if (d3 >= 0 && d4 <= d3) {                   /* vertex region b */
            w1 = 1; w2 = 0;
        } else {
            double vc = d1 * d4 - d3 * d2;
            if (vc <= 0 && d1 >= 0 && d3 <= 0) {     /* edge region ab */
                w1 = d1 / (d1 - d3); w2 = 0;
            } else {
                double cp[3];
                for (int i = 0; i < 3; ++i) cp[i] = p[i] - c[i];
                double d5 = dot3(ab, cp), d6 = dot3(ac, cp);
                if (d6 >= 0 && d5 <= d6) {           /* vertex region c */
                    w1 = 0; w2 = 1;
                } else {
                    double vb = d5 * d2 - d1 * d6;
                    if (vb <= 0 && d2 >= 0 && d6 <= 0) {   /* edge region ac */
                        w1 = 0; w2 = d2 / (d2 - d6);
                    } else {
                        double va = d3 * d6 - d5 * d4;
                        if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0) {  /* edge region bc */
                            double t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
                            w1 = 1 - t; w2 = t;
                        } else {                      /* face region */
                            double denom = 1.0 / (va + vb + vc);
                            w1 = vb * denom; w2 = vc * denom;
                        }
                    }
                }
            }
        }
    }
    for (int i = 0; i < 3; ++i) xbar[i] = a[i] + w1 * ab[i] + w2 * ac[i];
    bary[0] = w1;
    bary[1] = w2;
    double dd = 0;
    for (int i = 0; i < 3; ++i) { double t = p[i] - xbar[i]; dd += t * t; }
    return dd;
}

/* DistanceToBoundary (Algorithm 1): brute force over every element (every
 * Dirichlet element when the scene has a Neumann part).  Ties go to the
 * smaller element index (strict < keeps the first minimum). */
static double closest_point(const oracle_scene* s, const double* p, double* xbar, int* e_out, double* bary) {
    double best = INFINITY;
    int best_e = -1;
    double bx[3] = {0, 0, 0}, bb[2] = {0, 0};
    for (int e = 0; e < s->n_elem; ++e) {
        if (s->neumann && s->neumann[e]) continue;
        double xb[3] = {0, 0, 0}, b2[2];
        double d2;
        if (s->dim == 2) {
            const int* el = s->elem + 2 * e;
            d2 = closest_on_segment(p, s->vert + 2 * el[0], s->vert + 2 * el[1], xb, b2);
        } else {
            const int* el = s->elem + 3 * e;
            d2 = closest_on_triangle(p, s->vert + 3 * el[0], s->vert + 3 * el[1], s->vert + 3 * el[2], xb, b2);
        }
        if (d2 < best) {
            best = d2; best_e = e;
            bx[0] = xb[0]; bx[1] = xb[1]; bx[2] = xb[2];
            bb[0] = b2[0]; bb[1] = b2[1];
        }
    }
    for (int i = 0; i < s->dim; ++i) xbar[i] = bx[i];
    bary[0] = bb[0];
    bary[1] = bb[1];
    *e_out = best_e;
    return std::sqrt(best);
}

int oracle_closest_point(const oracle_scene* s, int n, const double* p, double* dist,
                         double* xbar, int* elem, double* bary) {
    for (int i = 0; i < n; ++i) {
        double xb[3], b2[2];
        int e;
        dist[i] = closest_point(s, p + (size_t)i * s->dim, xb, &e, b2);
        for (int k = 0; k < s->dim; ++k) xbar[(size_t)i * s->dim + k] = xb[k];
        elem[i] = e;
        bary[2 * (size_t)i] = b2[0];
        bary[2 * (size_t)i + 1] = b2[1];
    }
    return 0;
}

/* Weights of the element's vertices at barycentric point (bary). */
static void vertex_weights(int dim, const double* bary, double* w) {
    if (dim == 2) { w[0] = 1 - bary[0]; w[1] = bary[0]; w[2] = 0; }
    else { w[0] = 1 - bary[0] - bary[1]; w[1] = bary[0]; w[2] = bary[1]; }
}

/* Restricted field data g = c0 + c.x + x^T A x and its spatial gradient. */
static double field_value(const oracle_scene* s, const double* x, double* grad) {
    const double* c = s->field;
    double X[3] = {x[0], x[1], s->dim == 3 ? x[2] : 0.0};
    double A[3][3] = {{c[4], c[7], c[8]}, {c[7], c[5], c[9]}, {c[8], c[9], c[6]}};
    double g = c[0];
    for (int i = 0; i < 3; ++i) {
        g += c[1 + i] * X[i];
        double Ax = 0;
        for (int j = 0; j < 3; ++j) Ax += A[i][j] * X[j];
        g += X[i] * Ax;
        grad[i] = c[1 + i] + 2 * Ax;
    }
    return g;
}

/* Dirichlet value g at a boundary point. */
static double dirichlet_value(const oracle_scene* s, int e, const double* bary, const double* xbar) {
    if (s->data_kind == 1) {
        double grad[3];
        return field_value(s, xbar, grad);
    }
    double w[3];
    vertex_weights(s->dim, bary, w);
    const int* el = s->elem + (size_t)s->dim * e;
    double g = 0;
    for (int i = 0; i < s->dim; ++i) g += w[i] * s->g_vert[el[i]];
    return g;
}

/* Geometric unit normal of element e (unoriented). */
static void element_normal(const oracle_scene* s, int e, double* n) {
    const int* el = s->elem + (size_t)s->dim * e;
    if (s->dim == 2) {
        const double* a = s->vert + 2 * el[0];
        const double* b = s->vert + 2 * el[1];
        double tx = b[0] - a[0], ty = b[1] - a[1];
        double L = std::sqrt(tx * tx + ty * ty);
        n[0] = ty / L; n[1] = -tx / L; n[2] = 0;
    } else {
        const double* a = s->vert + 3 * el[0];
        const double* b = s->vert + 3 * el[1];
        const double* c = s->vert + 3 * el[2];
        double u[3], v[3];
        for (int i = 0; i < 3; ++i) { u[i] = b[i] - a[i]; v[i] = c[i] - a[i]; }
        double cr[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        double L = std::sqrt(dot3(cr, cr));
        for (int i = 0; i < 3; ++i) n[i] = cr[i] / L;
    }
}

/* Tangential gradient of the linearly interpolated vertex data on element e. */
static void surface_gradient(const oracle_scene* s, int e, double* grad) {
    const int* el = s->elem + (size_t)s->dim * e;
    grad[0] = grad[1] = grad[2] = 0;
    if (s->dim == 2) {
        const double* a = s->vert + 2 * el[0];
        const double* b = s->vert + 2 * el[1];
        double tx = b[0] - a[0], ty = b[1] - a[1];
        double L2 = tx * tx + ty * ty;
        double dg = s->g_vert[el[1]] - s->g_vert[el[0]];
        grad[0] = dg * tx / L2;
        grad[1] = dg * ty / L2;
    } else {
        const double* a = s->vert + 3 * el[0];
        const double* b = s->vert + 3 * el[1];
        const double* c = s->vert + 3 * el[2];
        double e1[3], e2[3];
        for (int i = 0; i < 3; ++i) { e1[i] = b[i] - a[i]; e2[i] = c[i] - a[i]; }
        double g11 = dot3(e1, e1), g12 = dot3(e1, e2), g22 = dot3(e2, e2);
        double det = g11 * g22 - g12 * g12;
        double r1 = s->g_vert[el[1]] - s->g_vert[el[0]];
        double r2 = s->g_vert[el[2]] - s->g_vert[el[0]];
        /* coefficients of grad in the (e1, e2) basis: G^{-1} (r1, r2) */
        double a1 = (g22 * r1 - g12 * r2) / det;
        double a2 = (-g12 * r1 + g11 * r2) / det;
        for (int i = 0; i < 3; ++i) grad[i] = a1 * e1[i] + a2 * e2[i];
    }
}

/* Recursive weight alpha = P(d) |dB(d)| of Algorithm 1, line "alpha <- P / p". */
double oracle_alpha(int dim, double sigma, double d) {
    if (sigma <= 0) return 1.0;
    double kd = std::sqrt(sigma) * d;
    if (dim == 2) return 1.0 / std::cyl_bessel_i(0.0, kd);
    return kd / std::sinh(kd);
}

/* The modified Bessel function K0 from the C++17 special-function library. */
double oracle_bessel_k0(double x) { return std::cyl_bessel_k(0.0, x); }

/* |B(d)| * G_d(r) with r = rho * d: the source weight of Algorithm 1 per unit f. */
double oracle_source_weight(int dim, double sigma, double d, double rho) {
    double r = rho * d;
    if (dim == 2) {
        double vol = kPi * d * d;
        double G;
        if (sigma <= 0) {
            G = std::log(d / r) / (2 * kPi);
        } else {
            double k = std::sqrt(sigma);
            G = (std::cyl_bessel_k(0.0, k * r)
                 - std::cyl_bessel_k(0.0, k * d) * std::cyl_bessel_i(0.0, k * r) / std::cyl_bessel_i(0.0, k * d))
                / (2 * kPi);
        }
        return vol * G;
    }
    double vol = 4.0 / 3.0 * kPi * d * d * d;
    double G;
    if (sigma <= 0) {
        G = (1.0 / r - 1.0 / d) / (4 * kPi);
    } else {
        double k = std::sqrt(sigma);
        G = std::sinh(k * (d - r)) / (4 * kPi * r * std::sinh(k * d));
    }
    return vol * G;
}

/* Gradient of a solution of -Lap u + sigma u = 0 at the centre of a ball of
 * radius R from its values on the sphere: grad u(c) = F E[n_y u(y)], y
 * uniform.  Writing u's l = 1 part as f(r) cos t, the gradient at c is f'(0)
 * and E[n_y u(y)] = f(R) / d; with f = I1(k r) (2D) or i1(k r) = (k r cosh k r
 * - sinh k r) / (k r)^2 (3D), f'(0) = k / d, so F = k / f(R); sigma = 0 gives
 * F = d / R (the mean-value property). */
double oracle_gradient_factor(int dim, double sigma, double R) {
    if (sigma <= 0) return dim / R;
    double k = std::sqrt(sigma), z = k * R;
    if (dim == 2) return k / std::cyl_bessel_i(1.0, z);
    double i1 = z < 1e-2 ? z / 3 + z * z * z / 30 + std::pow(z, 5) / 840
                         : (z * std::cosh(z) - std::sinh(z)) / (z * z);
    return k / i1;
}

/* Uniform direction on the unit circle / sphere and uniform point in the ball. */
static void sample_sphere(int dim, const Draws& r, double* w) {
    if (dim == 2) {
        double t = 2 * kPi * r.u[0];
        w[0] = std::cos(t); w[1] = std::sin(t); w[2] = 0;
    } else {
        double z = 1 - 2 * r.u[0];
        double st = 2 * std::sqrt(r.u[0] * (1 - r.u[0]));
        double ph = 2 * kPi * r.u[1];
        w[0] = st * std::cos(ph); w[1] = st * std::sin(ph); w[2] = z;
    }
}

static double sample_ball_radius(int dim, const Draws& r) {
    return dim == 2 ? std::sqrt(r.u[2]) : std::cbrt(r.u[2]);
}

struct PhaseResult {
    double x1[3];      /* point after the first sphere step (NaN if the walk never moved) */
    double u;          /* estimate from this phase */
    int kind;          /* KIND_* */
    int steps;         /* distance queries */
    int e;             /* terminal element */
    double bary[2];
    double xbar[3];
    double x_last[3];  /* walk point at termination */
    double ball_w;     /* ball-gradient weight F(R) (omega . n) of the first move, 0 if none */
    int on, on2;       /* walk on stars: the Neumann sides the walk sat on when it ended (-1: none) */
    double n_on[3], n2[3];   /* their normals, out of the domain */
};

/* The step's ball keeps a clearance of 1e-3 eps from the Dirichlet part: any
 * ball inside the domain gives an unbiased step, and the clearance keeps the
 * walk's landing points, computed in FP32 on the GPU, on the domain's side of
 * the boundary by more than rounding, which decides the orientation of the
 * boundary normal where the walk ends (away from its last point). */
static double step_radius(const oracle_scene* s, double d) { return d - 1e-3 * s->eps; }

/* Algorithm 1 (WalkOnSpheres) with Russian roulette, iterated instead of
 * recursed.  acc collects the source estimates S of every step.  With
 * ball_n (the ball-gradient estimator of Eq. dudn_mc_estimate at x0) the
 * first move is the gradient sample: no source, no roulette, and the weight
 * F(R) (omega . ball_n) is returned with the walk's estimate at y. */
static PhaseResult forward_walk(const oracle_scene* s, const double* x0, uint64_t walk_id, uint32_t phase,
                                const double* ball_n = NULL) {
    PhaseResult res;
    res.x1[0] = res.x1[1] = res.x1[2] = NAN;
    res.ball_w = 0;
    res.on = res.on2 = -1;
    double x[3] = {x0[0], x0[1], s->dim == 3 ? x0[2] : 0.0};
    double acc = 0;
    for (int k = 0;; ++k) {
        double xbar[3] = {0, 0, 0}, bary[2];
        int e;
        double d = closest_point(s, x, xbar, &e, bary);
        bool shell = d < s->eps;
        if (shell || k + 1 >= s->max_steps) {
            res.u = acc + dirichlet_value(s, e, bary, xbar);
            res.kind = shell ? KIND_SHELL : KIND_CAPPED;
            res.steps = k + 1;
            res.e = e;
            res.bary[0] = bary[0]; res.bary[1] = bary[1];
            for (int i = 0; i < 3; ++i) { res.xbar[i] = xbar[i]; res.x_last[i] = x[i]; }
            return res;
        }
        const bool ball = ball_n && k == 0;
        const double R = step_radius(s, d);
        if (s->f != 0 && !ball) {
            Draws rb = draw(s->seed_lo, s->seed_hi, walk_id, (uint32_t)k, phase, 1);
            double rho = sample_ball_radius(s->dim, rb);
            acc += oracle_source_weight(s->dim, s->sigma, R, rho) * s->f;
        }
        Draws r0 = draw(s->seed_lo, s->seed_hi, walk_id, (uint32_t)k, phase, 0);
        double alpha = oracle_alpha(s->dim, s->sigma, R);
        if (!ball && alpha < r0.u[2]) {
            res.u = acc;
            res.kind = KIND_ROULETTE;
            res.steps = k + 1;
            res.e = -1;
            res.bary[0] = res.bary[1] = 0;
            for (int i = 0; i < 3; ++i) { res.xbar[i] = 0; res.x_last[i] = x[i]; }
            return res;
        }
        double w[3];
        sample_sphere(s->dim, r0, w);
        for (int i = 0; i < s->dim; ++i) x[i] += R * w[i];
        if (ball) {
            double on = 0;
            for (int i = 0; i < s->dim; ++i) on += w[i] * ball_n[i];
            res.ball_w = oracle_gradient_factor(s->dim, s->sigma, R) * on;
        }
        if (k == 0) for (int i = 0; i < 3; ++i) res.x1[i] = i < s->dim ? x[i] : 0.0;
    }
}

/* ---------------------------------------------------------------------------
 * Walk on stars for a boundary split into a Dirichlet part and a reflecting
 * Neumann part (Sec. 3.4, Eq. mixed_bvp with Robin coefficient 0 and zero
 * Neumann data; the estimator of Walk on Stars, Sawhney et al. 2023, restated
 * here).  From a point x the walk uses the star-shaped region St(x, R): the
 * points of the ball B(x, R) that x sees without crossing the Neumann part.
 * R must keep St free of Dirichlet boundary (R <= distance to it) and every
 * ray from x must cross the Neumann part at most once inside B(x, R), which
 * holds when R is at most the distance to the closest silhouette point of the
 * Neumann part seen from x: a point where a ray from x grazes it (a vertex
 * whose two segments lie on the same side of the ray in 2D; an edge whose two
 * triangles lie on the same side of the plane through x and the edge in 3D)
 * or where it ends; where the part runs straight on through a vertex (flat
 * across an edge) it has none (runs_straight_on).  The radius is
 * R = max(min(d_D - c, d_sil), eps - c)
 * with the Dirichlet clearance c = 1e-3 eps of step_radius.  At the other
 * vertices (edges) a side test whose cross product (triple product in 3D) is
 * within a relative 1e-4 of zero counts as collinear (coplanar): both sides
 * collinear, no silhouette; one collinear and the other turning away, a
 * silhouette (seen from a point on the line of one side of a corner).  Seen
 * from a walk sitting on an element, that element's own vertices are
 * collinear (coplanar) with the walk's point by definition.
 * A ray meets an element where its barycentric coordinates lie within 1e-5
 * of the element (so that no ray slips between two neighbours), except a
 * neighbour of the side the walk sits on that lies behind that side's plane
 * (behind_side): a ray from the side into the domain cannot reach it, and
 * the tolerance would otherwise let a ray that grazes a reflex corner "hit"
 * the far side at its end, from the wrong side.  Nor does a ray from the side
 * cross an element on the side's own line (plane) through the walk's point
 * (coplanar_side): a direction nearly along the line would meet it at an
 * arbitrary t and take its normal's orientation from rounding.  A crossing up
 * to a relative 1e-5 plus 1e-4 eps beyond the ray's length counts, at the
 * ray's end: where the sphere of radius R meets
 * the Neumann part (it passes through the silhouette point that bounds R) a
 * direction that ends there lands on the boundary, and the walk must know.
 * Likewise a move from the Neumann part that hits nothing and leaves it by at
 * most 1e-4 eps along its normal (a direction nearly tangent to it) leaves the
 * walk on that element.  A walk that hits an element while it is still on
 * the side it left (within 1e-4 eps of it) sits on the edge (corner in 2D)
 * of the two: until it leaves either, its rays skip both and its directions
 * are turned into the wedge they bound (turn_inward).  Without this, a walk
 * that rounding puts exactly on a convex edge would leave through the side it
 * no longer tracks, from a start on that side's plane (a crossing at t = 0,
 * which no ray test counts).  The offset
 * point xbar - h n of the differential walk is mirrored across the Neumann
 * part where the segment from xbar to it crosses that part (next to a
 * Dirichlet-Neumann junction): across a reflecting boundary u extends evenly.
 * Where the main walk ended on the Neumann part and the offset point lies on
 * the same side (within 1e-4 eps of its plane, as the move from the end point
 * to the offset point is along it next to a right-angled junction), the
 * nested walks start on that side (and edge), as the main walk would.
 * One step: a direction v uniform on the sphere (reflected into the inward
 * half-space when x lies on the Neumann part), the ray x + t v up to the first
 * Neumann hit within R; the walk moves to the hit point (and is then on the
 * Neumann part) or to x + R v.  Its weight is the Poisson kernel of the ball
 * at that distance per unit solid angle, |S^(d-1)| t^(d-1) |G_R'(t)| with
 * G_R the ball's Green's function: 1 for sigma = 0 and alpha(R) at t = R, so
 * Russian roulette uses it as the survival probability.  The source term
 * samples a point of the ball as in Algorithm 1 and counts it only if x sees
 * it.  The walk ends in the eps-shell of the Dirichlet part.
 * ------------------------------------------------------------------------- */
struct Adjacency {
    /* per element and per endpoint (2D) / per edge ab, bc, ca (3D): the vertex of the
       Neumann neighbour across it (its other vertex / the vertex opposite the shared
       edge), -1 where the Neumann part ends */
    std::vector<int> other;
};

static Adjacency build_adjacency(const oracle_scene* s) {
    Adjacency a;
    a.other.assign((size_t)s->n_elem * s->dim, -1);
    if (!s->neumann) return a;
    if (s->dim == 2) {
        std::map<int, std::vector<int>> at;     /* vertex -> Neumann segments containing it */
        for (int e = 0; e < s->n_elem; ++e)
            if (s->neumann[e]) for (int j = 0; j < 2; ++j) at[s->elem[2 * e + j]].push_back(e);
        for (int e = 0; e < s->n_elem; ++e) {
            if (!s->neumann[e]) continue;
            for (int j = 0; j < 2; ++j) {
                const int v = s->elem[2 * e + j];
                for (int f : at[v])
                    if (f != e) { a.other[2 * (size_t)e + j] = s->elem[2 * f] == v ? s->elem[2 * f + 1] : s->elem[2 * f]; break; }
            }
        }
    } else {
        std::map<std::pair<int, int>, std::vector<int>> at;   /* edge -> Neumann triangles containing it */
        auto key = [](int p, int q) { return p < q ? std::make_pair(p, q) : std::make_pair(q, p); };
        for (int e = 0; e < s->n_elem; ++e) {
            if (!s->neumann[e]) continue;
            const int* t = s->elem + 3 * e;
            for (int j = 0; j < 3; ++j) at[key(t[j], t[(j + 1) % 3])].push_back(e);
        }
        for (int e = 0; e < s->n_elem; ++e) {
            if (!s->neumann[e]) continue;
            const int* t = s->elem + 3 * e;
            for (int j = 0; j < 3; ++j) {
                for (int f : at[key(t[j], t[(j + 1) % 3])]) {
                    if (f == e) continue;
                    const int* u = s->elem + 3 * f;
                    for (int i = 0; i < 3; ++i)
                        if (u[i] != t[j] && u[i] != t[(j + 1) % 3]) a.other[3 * (size_t)e + j] = u[i];
                    break;
                }
            }
        }
    }
    return a;
}

static double cross2(const double* a, const double* b) { return a[0] * b[1] - a[1] * b[0]; }

/* Silhouette rule from the two side tests s1, s2 and their scales m1, m2 (the
 * products of the lengths involved): a side test within a relative 1e-4 of
 * zero counts as collinear / coplanar. */
static bool silhouette_rule(double s1, double m1, double s2, double m2) {
    const bool c1 = std::fabs(s1) <= 1e-4 * m1, c2 = std::fabs(s2) <= 1e-4 * m2;
    if (c1 && c2) return false;      /* the boundary runs straight on through it */
    if (c1 || c2) return true;       /* one side along the line of sight, the other turns */
    return s1 * s2 > 0;              /* both neighbours on the same side */
}

static double det3(const double* a, const double* b, const double* c) {
    return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
}

/* Distance from x to the closest silhouette point of the Neumann part. */
/* Where the Neumann part runs straight on, it has no silhouette point from any
 * x: a vertex v between segments vw and vz whose unit directions w -> v and
 * v -> z agree within a relative 1e-6 (2D), or an edge ab between triangles
 * abc and abz whose unit normals (b - a) x (c - a) and (z - a) x (b - a)
 * agree within a relative 1e-6 (3D; c and z on opposite sides of ab). */
static bool runs_straight_on(int d, const double* a, const double* b, const double* c, const double* z) {
    if (d == 2) {   /* v = a, w = b, z: directions w -> v and v -> z */
        const double u1[3] = {a[0] - b[0], a[1] - b[1], 0}, u2[3] = {z[0] - a[0], z[1] - a[1], 0};
        return dot3(u1, u2) >= (1 - 1e-6) * std::sqrt(dot3(u1, u1) * dot3(u2, u2));
    }
    const double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const double ac[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    const double az[3] = {z[0] - a[0], z[1] - a[1], z[2] - a[2]};
    const double n1[3] = {ab[1] * ac[2] - ab[2] * ac[1], ab[2] * ac[0] - ab[0] * ac[2], ab[0] * ac[1] - ab[1] * ac[0]};
    const double n2[3] = {az[1] * ab[2] - az[2] * ab[1], az[2] * ab[0] - az[0] * ab[2], az[0] * ab[1] - az[1] * ab[0]};
    return dot3(n1, n2) >= (1 - 1e-6) * std::sqrt(dot3(n1, n1) * dot3(n2, n2));
}

/* True if element f (-1: none) has exactly the vertices p, q (and r in 3D). */
static bool element_is(const oracle_scene* s, int f, int p, int q, int r) {
    if (f < 0) return false;
    const int* el = s->elem + (size_t)s->dim * f;
    const int want[3] = {p, q, r};
    for (int i = 0; i < s->dim; ++i) {
        bool found = false;
        for (int j = 0; j < s->dim; ++j) found = found || el[j] == want[i];
        if (!found) return false;
    }
    return true;
}

/* The walk sits on element `on` (and `on2` at an edge; -1: none): x lies on
 * them, so a side test of the silhouette rule whose three points (x, the
 * site's vertex / edge and the other vertex) span one of them is zero by
 * definition, whatever the arithmetic gives. */
static double silhouette_distance(const oracle_scene* s, const Adjacency& adj, const double* x, int on, int on2) {
    double best = INFINITY;
    const int d = s->dim;
    for (int e = 0; e < s->n_elem; ++e) {
        if (!s->neumann[e]) continue;
        const int* el = s->elem + (size_t)d * e;
        if (d == 2) {
            for (int j = 0; j < 2; ++j) {
                const double* v = s->vert + 2 * el[j];
                const double* w = s->vert + 2 * el[1 - j];
                const int nb = adj.other[2 * (size_t)e + j];
                if (nb >= 0 && runs_straight_on(2, v, w, NULL, s->vert + 2 * nb)) continue;
                const double rv[2] = {v[0] - x[0], v[1] - x[1]};
                bool sil = nb < 0;
                if (!sil) {
                    const double* z = s->vert + 2 * nb;
                    const double rw[2] = {w[0] - x[0], w[1] - x[1]}, rz[2] = {z[0] - x[0], z[1] - x[1]};
                    const double lv = std::hypot(rv[0], rv[1]);
                    const bool own1 = e == on || e == on2;
                    const bool own2 = element_is(s, on, el[j], nb, -1) || element_is(s, on2, el[j], nb, -1);
                    sil = silhouette_rule(own1 ? 0.0 : cross2(rv, rw), lv * std::hypot(rw[0], rw[1]),
                                          own2 ? 0.0 : cross2(rv, rz), lv * std::hypot(rz[0], rz[1]));
                }
                if (sil) best = std::min(best, std::sqrt(rv[0] * rv[0] + rv[1] * rv[1]));
            }
        } else {
            for (int j = 0; j < 3; ++j) {
                const double* a = s->vert + 3 * el[j];
                const double* b = s->vert + 3 * el[(j + 1) % 3];
                const double* c = s->vert + 3 * el[(j + 2) % 3];
                const int nb = adj.other[3 * (size_t)e + j];
                if (nb >= 0 && runs_straight_on(3, a, b, c, s->vert + 3 * nb)) continue;
                const double ra[3] = {a[0] - x[0], a[1] - x[1], a[2] - x[2]};
                const double rb[3] = {b[0] - x[0], b[1] - x[1], b[2] - x[2]};
                bool sil = nb < 0;
                if (!sil) {
                    const double* z = s->vert + 3 * nb;
                    const double rc[3] = {c[0] - x[0], c[1] - x[1], c[2] - x[2]};
                    const double rz[3] = {z[0] - x[0], z[1] - x[1], z[2] - x[2]};
                    const double n[3] = {ra[1] * rb[2] - ra[2] * rb[1], ra[2] * rb[0] - ra[0] * rb[2],
                                         ra[0] * rb[1] - ra[1] * rb[0]};
                    const double ln = std::sqrt(dot3(n, n));
                    const bool own1 = e == on || e == on2;
                    const int ia = el[j], ib = el[(j + 1) % 3];
                    const bool own2 = element_is(s, on, ia, ib, nb) || element_is(s, on2, ia, ib, nb);
                    sil = silhouette_rule(own1 ? 0.0 : det3(ra, rb, rc), ln * std::sqrt(dot3(rc, rc)),
                                          own2 ? 0.0 : det3(ra, rb, rz), ln * std::sqrt(dot3(rz, rz)));
                }
                if (!sil) continue;
                /* distance from x to the segment ab */
                const double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
                const double len2 = dot3(ab, ab);
                double t = len2 > 0 ? -dot3(ra, ab) / len2 : 0.0;
                t = std::min(1.0, std::max(0.0, t));
                double off[3];
                for (int i = 0; i < 3; ++i) off[i] = a[i] + t * ab[i] - x[i];
                best = std::min(best, std::sqrt(dot3(off, off)));
            }
        }
    }
    return best;
}

/* True if elements e and f share a vertex. */
static bool share_vertex(const oracle_scene* s, int e, int f) {
    const int* a = s->elem + (size_t)s->dim * e;
    const int* b = s->elem + (size_t)s->dim * f;
    for (int i = 0; i < s->dim; ++i)
        for (int j = 0; j < s->dim; ++j)
            if (a[i] == b[j]) return true;
    return false;
}

/* Element f lies behind side e (unit normal n_e, out of the domain): f
 * shares a vertex with e and none of its vertices lies in front of e's line
 * (plane), up to a relative 1e-6: (p - a) . n_e >= -1e-6 |p - a| for every
 * vertex p of f, a e's first vertex.  Flat continuations of e and the far
 * side of a reflex corner are behind it; a ray from e into the domain cannot
 * reach them. */
static bool behind_side(const oracle_scene* s, int e, const double* n_e, int f) {
    if (!share_vertex(s, e, f)) return false;
    const int d = s->dim;
    const double* a = s->vert + (size_t)d * s->elem[(size_t)d * e];
    for (int j = 0; j < d; ++j) {
        const double* p = s->vert + (size_t)d * s->elem[(size_t)d * f + j];
        double r[3] = {0, 0, 0};
        for (int i = 0; i < d; ++i) r[i] = p[i] - a[i];
        if (dot3(r, n_e) < -1e-6 * std::sqrt(dot3(r, r))) return false;
    }
    return true;
}

/* Element f lies on the line (plane) of side e (unit normal n_e) through x:
 * their normals are parallel within a relative 1e-6 and f's line (plane)
 * passes within 1e-4 eps of x.  A ray from x does not cross it, whatever
 * rounding makes of t (a direction nearly along the line meets f's line at
 * an arbitrary t). */
static bool coplanar_side(const oracle_scene* s, const double* x, const double* n_e, int f) {
    double m[3];
    element_normal(s, f, m);
    if (std::fabs(dot3(m, n_e)) < 1 - 1e-6) return false;
    const double* a = s->vert + (size_t)s->dim * s->elem[(size_t)s->dim * f];
    double r[3] = {0, 0, 0};
    for (int i = 0; i < s->dim; ++i) r[i] = x[i] - a[i];
    return std::fabs(dot3(r, m)) <= 1e-4 * s->eps;
}

/* A ray from the side e (the walk sits on it) does not hit f. */
static bool skipped_from(const oracle_scene* s, const double* x, int e, const double* n_e, int f) {
    return e >= 0 && (behind_side(s, e, n_e, f) || coplanar_side(s, x, n_e, f));
}

/* First crossing of the ray x + t v (0 < t < tmax (1 + 1e-5) + slack) with a
 * Neumann element other than `skip` and `skip2` (the sides the walk sits on,
 * with their normals n_skip, n_skip2 out of the domain), the elements behind
 * them and those on their lines (planes) through x; returns min(t, tmax)
 * (tmax if none) and the element (-1 if none). */
static double ray_neumann(const oracle_scene* s, const double* x, const double* v, double tmax, int skip,
                          const double* n_skip, int skip2, const double* n_skip2, double slack, int* e_out) {
    double best = INFINITY;
    *e_out = -1;
    for (int e = 0; e < s->n_elem; ++e) {
        if (!s->neumann[e] || e == skip || e == skip2) continue;
        const int* el = s->elem + (size_t)s->dim * e;
        double t;
        if (s->dim == 2) {
            const double* a = s->vert + 2 * el[0];
            const double* b = s->vert + 2 * el[1];
            const double ab[2] = {b[0] - a[0], b[1] - a[1]}, ax[2] = {a[0] - x[0], a[1] - x[1]};
            const double den = cross2(v, ab);
            if (den == 0) continue;
            t = cross2(ax, ab) / den;
            const double u = cross2(ax, v) / den;
            if (!(u >= -1e-5 && u <= 1 + 1e-5)) continue;
        } else {
            const double* a = s->vert + 3 * el[0];
            const double* b = s->vert + 3 * el[1];
            const double* c = s->vert + 3 * el[2];
            double e1[3], e2[3], tv[3];
            for (int i = 0; i < 3; ++i) { e1[i] = b[i] - a[i]; e2[i] = c[i] - a[i]; tv[i] = x[i] - a[i]; }
            const double p[3] = {v[1] * e2[2] - v[2] * e2[1], v[2] * e2[0] - v[0] * e2[2], v[0] * e2[1] - v[1] * e2[0]};
            const double det = dot3(e1, p);
            if (det == 0) continue;
            const double u = dot3(tv, p) / det;
            if (!(u >= -1e-5 && u <= 1 + 1e-5)) continue;
            const double q[3] = {tv[1] * e1[2] - tv[2] * e1[1], tv[2] * e1[0] - tv[0] * e1[2], tv[0] * e1[1] - tv[1] * e1[0]};
            const double w = dot3(v, q) / det;
            if (!(w >= -1e-5 && u + w <= 1 + 1e-5)) continue;
            t = dot3(e2, q) / det;
        }
        if (!(t > 0 && t < tmax * (1 + 1e-5) + slack && t < best)) continue;
        if (skipped_from(s, x, skip, n_skip, e) || skipped_from(s, x, skip2, n_skip2, e)) continue;
        best = t;
        *e_out = e;
    }
    return std::min(best, tmax);
}

/* Survival weight of a star step of length t inside the ball of radius R:
 * |S^(d-1)| t^(d-1) |G_R'(t)| for the screened ball Green's function G_R. */
double oracle_star_weight(int dim, double sigma, double t, double R) {
    if (sigma <= 0) return 1.0;
    const double k = std::sqrt(sigma);
    if (dim == 2)
        return k * t * (std::cyl_bessel_k(1.0, k * t)
                        + std::cyl_bessel_i(1.0, k * t) * std::cyl_bessel_k(0.0, k * R) / std::cyl_bessel_i(0.0, k * R));
    return (k * t * std::cosh(k * (R - t)) + std::sinh(k * (R - t))) / std::sinh(k * R);
}

/* A direction drawn at a point of the Neumann part is turned into the
 * domain: into the inner half-space of the side the walk sits on (n_on, out
 * of the domain) by v -> -v; at an edge, where the walk also lies on a second
 * side (n2), by mirrors across the plane it still points out of, alternately,
 * at most 4 (a ray in a wedge of interior angle a turns inward after at most
 * ceil(pi / a) mirrors: any edge of 45 degrees or more).  At a right-angled
 * edge this makes the direction uniform over the quarter-space. */
static void turn_inward(double* v, int on, const double* n_on, int on2, const double* n2) {
    if (on >= 0 && dot3(v, n_on) > 0) for (int i = 0; i < 3; ++i) v[i] = -v[i];
    if (on2 < 0) return;
    for (int m = 0; m < 4; ++m) {
        const double* n = dot3(v, n2) > 0 ? n2 : dot3(v, n_on) > 0 ? n_on : NULL;
        if (!n) return;
        const double c = 2 * dot3(v, n);
        for (int i = 0; i < 3; ++i) v[i] -= c * n[i];
    }
}

/* turn_inward for the tests: n directions v (n x 3, in place) with the sides'
 * normals n_on and n2 (n2 NULL: on one side only). */
void oracle_turn_inward(int n, double* v, const double* n_on, const double* n2) {
    for (int i = 0; i < n; ++i) turn_inward(v + 3 * (size_t)i, 0, n_on, n2 ? 0 : -1, n2 ? n2 : n_on);
}

/* ray_neumann for the tests: the first Neumann crossing of x + t v within
 * tmax for a walk on sides `skip` (normal n_skip) and `skip2` (n_skip2; -1 /
 * NULL: none), with the walk's slack of 1e-4 eps.  Returns t, the element in
 * *e_out. */
double oracle_ray_neumann(const oracle_scene* s, const double* x, const double* v, double tmax, int skip,
                          const double* n_skip, int skip2, const double* n_skip2, int* e_out) {
    return ray_neumann(s, x, v, tmax, skip, n_skip, skip2, n_skip2, 1e-4 * s->eps, e_out);
}

/* Length (2D) or area (3D) of element e. */
static double element_measure(const oracle_scene* s, int e) {
    const int d = s->dim;
    const int* el = s->elem + (size_t)d * e;
    const double* a = s->vert + (size_t)d * el[0];
    const double* b = s->vert + (size_t)d * el[1];
    if (d == 2) return std::hypot(b[0] - a[0], b[1] - a[1]);
    const double* c = s->vert + (size_t)d * el[2];
    double u[3], v[3];
    for (int i = 0; i < 3; ++i) { u[i] = b[i] - a[i]; v[i] = c[i] - a[i]; }
    const double w[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    return 0.5 * std::sqrt(dot3(w, w));
}

/* The ball's Green's function G_R(t) at distance t from the centre (the source
 * weight above divided by the ball's volume). */
static double ball_green(int dim, double sigma, double t, double R) {
    const double vol = dim == 2 ? kPi * R * R : 4.0 / 3.0 * kPi * R * R * R;
    return oracle_source_weight(dim, sigma, R, t / R) / vol;
}

/* The 32-bit finaliser of Appleby's MurmurHash3: a bijection of 32-bit words
 * in which every input bit reaches every output bit. */
static uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

/* Uniform in (0, 1) for the Neumann element of index c (counted among the
 * Neumann elements in input order), from the step's word w (word 2 of block 2):
 * fmix32(w + (c + 1) * 0x9E3779B9).  For each c it is uniform over w (fmix32 is a
 * bijection); the mix spreads neighbouring indices apart. */
static double element_uniform(uint32_t w, int c) {
    return to_uniform(fmix32(w + (uint32_t)(c + 1) * 0x9E3779B9u));
}

/* Element e lies wholly behind side `side` (unit normal n out of the domain)
 * of a walk at x: every vertex more than 2e-4 eps behind the side's plane
 * through x.  x sees no point of it. */
static bool wholly_behind(const oracle_scene* s, int e, const double* x, int side, const double* n) {
    if (side < 0) return false;
    const int d = s->dim;
    for (int j = 0; j < d; ++j) {
        const double* p = s->vert + (size_t)d * s->elem[(size_t)d * e + j];
        double r[3] = {0, 0, 0};
        for (int i = 0; i < d; ++i) r[i] = p[i] - x[i];
        if (!(dot3(r, n) > 2e-4 * s->eps)) return false;
    }
    return true;
}

/* The Neumann-data term of a walk-on-stars step (Sec. 3.4, Eq. mixed_bvp with
 * Robin coefficient 0 and data h = du/dn; Green's second identity on the star
 * St(x, R)): the walk adds (1 / a(x)) times the integral of G_R(x, z) h(z) over
 * the part of the Neumann boundary in the ball that x sees, a(x) the share of
 * the directions around x that point into the domain (1 inside, 1/2 on a
 * side, (pi - angle between the two normals) / 2 pi at an edge).  One sample:
 * every Neumann element closer to x than R (1 - 1e-4) and not wholly behind a
 * side the walk sits on (it would give 0) is a candidate, of total measure A (the margin leaves out the elements that only touch the ball
 * at a silhouette point, whose distance to x is R itself, and parts of others
 * within 1e-4 R of the sphere, where G_R is below 1e-4 of its size);
 * the element is drawn with probability proportional to its measure (the
 * candidate with the least -log(U_c) / |e_c|, U_c from element_uniform, so that
 * the draw does not depend on the order of the candidates), z uniformly on it
 * (block 2 of the step: words 0 and 1); the estimate is A G_R(|z - x|) h(e) / a(x) if |z - x| < R
 * and x sees z, else 0.  x sees z if z lies on a side the walk sits on, or
 * else, z not behind those sides (a point (z - x) . n > 1e-4 eps out of a
 * side's plane, or an element behind it by the ray rule, unless it is on the
 * side's plane), no Neumann element crosses the segment before 1 - 1e-4 of
 * its length (the ray rules of the step). */
static double neumann_data_sample(const oracle_scene* s, const double* x, double R, int on, const double* n_on,
                                  int on2, const double* n2, uint64_t walk_id, uint32_t k, uint32_t phase) {
    const int d = s->dim;
    const uint32_t ctr[4] = {(uint32_t)walk_id, (uint32_t)(walk_id >> 32), k, (phase << 8) | 2u};
    const uint32_t key2[2] = {s->seed_lo, s->seed_hi};
    uint32_t blk[4];
    philox4x32_10(ctr, key2, blk);
    double A = 0, best = INFINITY;
    int pick = -1;
    for (int e = 0, c = 0; e < s->n_elem; ++e) {
        if (!s->neumann[e]) continue;
        const int ci = c++;
        const int* el = s->elem + (size_t)d * e;
        double xb[3] = {0, 0, 0}, b2[2];
        const double d2 = d == 2 ? closest_on_segment(x, s->vert + 2 * el[0], s->vert + 2 * el[1], xb, b2)
                                 : closest_on_triangle(x, s->vert + 3 * el[0], s->vert + 3 * el[1],
                                                       s->vert + 3 * el[2], xb, b2);
        if (!(d2 < (1 - 2e-4) * R * R)) continue;
        if (wholly_behind(s, e, x, on, n_on) || wholly_behind(s, e, x, on2, n2)) continue;
        const double m = element_measure(s, e);
        if (!(m > 0)) continue;
        A += m;
        const double key = -std::log(element_uniform(blk[2], ci)) / m;
        if (key < best) { best = key; pick = e; }
    }
    if (pick < 0) return 0;
    const Draws r = {{to_uniform(blk[0]), to_uniform(blk[1]), to_uniform(blk[2])}};
    const int* el = s->elem + (size_t)d * pick;
    double z[3] = {0, 0, 0};
    if (d == 2) {
        const double* a = s->vert + 2 * el[0];
        const double* b = s->vert + 2 * el[1];
        for (int i = 0; i < 2; ++i) z[i] = a[i] + r.u[0] * (b[i] - a[i]);
    } else {
        const double* a = s->vert + 3 * el[0];
        const double* b = s->vert + 3 * el[1];
        const double* c = s->vert + 3 * el[2];
        const double q = std::sqrt(r.u[0]);
        for (int i = 0; i < 3; ++i) z[i] = (1 - q) * a[i] + q * (1 - r.u[1]) * b[i] + q * r.u[1] * c[i];
    }
    double v[3] = {0, 0, 0};
    for (int i = 0; i < d; ++i) v[i] = z[i] - x[i];
    const double t = std::sqrt(dot3(v, v));
    if (!(t < R) || !(t > 0)) return 0;
    if (pick != on && pick != on2) {
        const double on_line = 1e-4 * s->eps;
        const int side[2] = {on, on2};
        const double* nrm[2] = {n_on, n2};
        for (int j = 0; j < 2; ++j) {
            if (side[j] < 0) continue;
            if (coplanar_side(s, x, nrm[j], pick)) continue;
            if (behind_side(s, side[j], nrm[j], pick) || dot3(v, nrm[j]) > on_line) return 0;
        }
        for (int i = 0; i < 3; ++i) v[i] /= t;
        int he;
        ray_neumann(s, x, v, t * (1 - 1e-4), on, n_on, on2, n2, 0.0, &he);
        if (he >= 0) return 0;
    }
    double share = 1;
    if (on2 >= 0) share = (kPi - std::acos(std::max(-1.0, std::min(1.0, dot3(n_on, n2))))) / (2 * kPi);
    else if (on >= 0) share = 0.5;
    return A * ball_green(d, s->sigma, t, R) * s->neumann_h[pick] / share;
}

/* neumann_data_sample for the tests: the Neumann-data term of one step from x
 * with radius R, for a walk on sides on / on2 (normals n_on / n2, -1 / NULL:
 * none), at step k of phase `phase` of walk walk_id. */
double oracle_neumann_data_sample(const oracle_scene* s, const double* x, double R, int on, const double* n_on,
                                  int on2, const double* n2, uint64_t walk_id, uint32_t k, uint32_t phase) {
    const double zero[3] = {0, 0, 0};
    return neumann_data_sample(s, x, R, on, n_on ? n_on : zero, on2, n2 ? n2 : zero, walk_id, k, phase);
}

/* Where a walk on stars starts: the Neumann side it sits on (-1: inside) and,
 * on an edge, the second side, with their normals out of the domain. */
struct StarStart {
    int on = -1, on2 = -1;
    double n_on[3] = {0, 0, 0}, n2[3] = {0, 0, 0};
};

static PhaseResult wost_walk(const oracle_scene* s, const Adjacency& adj, const double* x0, uint64_t walk_id,
                             uint32_t phase, const StarStart& st) {
    PhaseResult res;
    res.x1[0] = res.x1[1] = res.x1[2] = NAN;
    res.ball_w = 0;
    const int d = s->dim;
    double x[3] = {x0[0], x0[1], d == 3 ? x0[2] : 0.0};
    double acc = 0;
    int on = st.on;                    /* the Neumann element the walk sits on, -1 inside */
    int on2 = st.on2;                  /* at an edge: the side it came from, still under it */
    double n_on[3], n2[3];             /* their normals, out of the domain */
    for (int i = 0; i < 3; ++i) { n_on[i] = st.n_on[i]; n2[i] = st.n2[i]; }
    const double on_line = 1e-4 * s->eps;
    for (int k = 0;; ++k) {
        double xbar[3] = {0, 0, 0}, bary[2];
        int e;
        const double dD = closest_point(s, x, xbar, &e, bary);
        const bool shell = dD < s->eps;
        if (shell || k + 1 >= s->max_steps) {
            res.u = acc + dirichlet_value(s, e, bary, xbar);
            res.kind = shell ? KIND_SHELL : KIND_CAPPED;
            res.steps = k + 1;
            res.e = e;
            res.bary[0] = bary[0]; res.bary[1] = bary[1];
            for (int i = 0; i < 3; ++i) { res.xbar[i] = xbar[i]; res.x_last[i] = x[i]; }
            res.on = on; res.on2 = on2;
            for (int i = 0; i < 3; ++i) { res.n_on[i] = n_on[i]; res.n2[i] = n2[i]; }
            return res;
        }
        const double R = std::max(std::min(step_radius(s, dD), silhouette_distance(s, adj, x, on, on2)), step_radius(s, s->eps));
        if (s->f != 0) {   /* source: a point of the ball, counted if x sees it */
            Draws rb = draw(s->seed_lo, s->seed_hi, walk_id, (uint32_t)k, phase, 1);
            double w[3];
            sample_sphere(d, rb, w);
            turn_inward(w, on, n_on, on2, n2);
            const double rho = sample_ball_radius(d, rb);
            int e2;
            ray_neumann(s, x, w, rho * R, on, n_on, on2, n2, on_line, &e2);
            if (e2 < 0) acc += oracle_source_weight(d, s->sigma, R, rho) * s->f;
        }
        if (s->neumann_h)   /* Neumann data: a point of the Neumann part in the ball, counted if x sees it */
            acc += neumann_data_sample(s, x, R, on, n_on, on2, n2, walk_id, (uint32_t)k, phase);
        Draws r0 = draw(s->seed_lo, s->seed_hi, walk_id, (uint32_t)k, phase, 0);
        double v[3];
        sample_sphere(d, r0, v);
        turn_inward(v, on, n_on, on2, n2);
        int he;
        const double t = ray_neumann(s, x, v, R, on, n_on, on2, n2, on_line, &he);
        if (oracle_star_weight(d, s->sigma, t, R) < r0.u[2]) {
            res.u = acc;
            res.kind = KIND_ROULETTE;
            res.steps = k + 1;
            res.e = -1;
            res.bary[0] = res.bary[1] = 0;
            for (int i = 0; i < 3; ++i) { res.xbar[i] = 0; res.x_last[i] = x[i]; }
            res.on = res.on2 = -1;
            return res;
        }
        for (int i = 0; i < d; ++i) x[i] += t * v[i];
        /* a move that leaves a side by at most 1e-4 eps along its normal (a
         * direction nearly tangent to it) leaves the walk on that side */
        const bool keep = on >= 0 && std::fabs(t * dot3(v, n_on)) <= on_line;
        const bool keep2 = on2 >= 0 && std::fabs(t * dot3(v, n2)) <= on_line;
        if (he >= 0) {   /* on the element hit; on an edge if still on the side it left */
            if (keep) { on2 = on; for (int i = 0; i < 3; ++i) n2[i] = n_on[i]; } else on2 = -1;
            on = he;
            element_normal(s, he, n_on);
            if (dot3(n_on, v) < 0) for (int i = 0; i < 3; ++i) n_on[i] = -n_on[i];
        } else if (keep) {
            if (!keep2) on2 = -1;
        } else if (keep2) {
            on = on2;
            for (int i = 0; i < 3; ++i) n_on[i] = n2[i];
            on2 = -1;
        } else {
            on = on2 = -1;
        }
        if (k == 0) for (int i = 0; i < 3; ++i) res.x1[i] = i < d ? x[i] : 0.0;
    }
}

/* A query point on the Neumann part (within 1e-3 eps of it) starts its walk
 * on the closest Neumann element (ties to the lower index), with that
 * element's normal oriented out of the domain: the point 1e-3 of the
 * element's size behind the element's centre is inside.  Returns the
 * element, or -1 for a point inside the domain. */
int oracle_inside(const oracle_scene* s, int n, const double* xq, int* inside);

static int neumann_start(const oracle_scene* s, const double* x0, double* n_out) {
    const int d = s->dim;
    double best = INFINITY;
    int best_e = -1;
    for (int e = 0; e < s->n_elem; ++e) {
        if (!s->neumann[e]) continue;
        double xb[3] = {0, 0, 0}, b2[2];
        const int* el = s->elem + (size_t)d * e;
        const double d2 = d == 2 ? closest_on_segment(x0, s->vert + 2 * el[0], s->vert + 2 * el[1], xb, b2)
                                 : closest_on_triangle(x0, s->vert + 3 * el[0], s->vert + 3 * el[1],
                                                       s->vert + 3 * el[2], xb, b2);
        if (d2 < best) { best = d2; best_e = e; }
    }
    if (best_e < 0 || std::sqrt(best) > 1e-3 * s->eps) return -1;
    double n[3];
    element_normal(s, best_e, n);
    const int* el = s->elem + (size_t)d * best_e;
    double c[3] = {0, 0, 0}, size;
    for (int j = 0; j < d; ++j)
        for (int i = 0; i < d; ++i) c[i] += s->vert[(size_t)d * el[j] + i] / d;
    if (d == 2) {
        size = std::hypot(s->vert[2 * el[1]] - s->vert[2 * el[0]], s->vert[2 * el[1] + 1] - s->vert[2 * el[0] + 1]);
    } else {
        double u[3], v[3], w[3];
        for (int i = 0; i < 3; ++i) { u[i] = s->vert[3 * el[1] + i] - s->vert[3 * el[0] + i];
                                      v[i] = s->vert[3 * el[2] + i] - s->vert[3 * el[0] + i]; }
        w[0] = u[1] * v[2] - u[2] * v[1]; w[1] = u[2] * v[0] - u[0] * v[2]; w[2] = u[0] * v[1] - u[1] * v[0];
        size = std::sqrt(std::sqrt(dot3(w, w)));
    }
    double behind[3];
    for (int i = 0; i < d; ++i) behind[i] = c[i] - 1e-3 * size * n[i];
    int in = 0;
    oracle_inside(s, 1, behind, &in);
    for (int i = 0; i < 3; ++i) n_out[i] = in ? n[i] : -n[i];
    return best_e;
}

/* One phase of a walk: walk on spheres, or walk on stars with a Neumann part
 * (the main walk of a query point on the Neumann part starts on it; a nested
 * walk starts where `nested` says). */
static PhaseResult phase_walk(const oracle_scene* s, const Adjacency* adj, const double* x0, uint64_t walk_id,
                              uint32_t phase, const double* ball_n, const StarStart* nested = NULL) {
    if (s->neumann) {
        StarStart st;
        if (phase == 0) st.on = neumann_start(s, x0, st.n_on);
        else if (nested) st = *nested;
        return wost_walk(s, *adj, x0, walk_id, phase, st);
    }
    return forward_walk(s, x0, walk_id, phase, ball_n);
}

/* Per-walk outputs; any pointer may be NULL. */
typedef struct {
    double* u_hat;     /* n: forward estimate of u at the query point */
    double* udot;      /* n * n_param: differential estimate */
    double* dudn;      /* n: (g(xbar) - mean nested u) / h */
    double* u_off;     /* n: mean of the nested walks */
    int* elem;         /* n: terminal element of the differential walk (-1: roulette) */
    double* bary;      /* n * 2 */
    double* normal;    /* n * 3 */
    double* xbar;      /* n * 3 */
    int* kind;         /* n * (K + 1) */
    int* steps;        /* n * (K + 1) */
    double* x1;        /* n * 3: main walk's point after its first step (NaN if none) */
    double* x_end;     /* n * 3: main walk's point where it stopped */
    double* u_plain;   /* n: mean of the nested estimates without the control variate */
    double* disp_n;    /* n: mean over the nested walks of n . (x_end - x_off) */
    double* disp_t;    /* n: mean over the nested walks of t . (x_end - x_off) (0 without a table) */
} oracle_walk_out;

/* Algorithm 2 (DiffWalkOnSpheres) extended, as Sec. 4.1 observation 2
 * describes, to also return u from the same path (source sum + g(xbar)).
 * With mode 0 only Algorithm 1 runs (no nested walks, no derivative). */
static void run_one(const oracle_scene* s, const Adjacency* adj, const double* x0, uint64_t walk_id, int mode,
                    const oracle_walk_out* o, size_t idx) {
    int P = s->n_param;
    int slots = s->K + 1;
    PhaseResult main = phase_walk(s, adj, x0, walk_id, 0, NULL);
    if (o->u_hat) o->u_hat[idx] = main.u;
    if (o->kind) { o->kind[idx * slots] = main.kind; }
    if (o->steps) { o->steps[idx * slots] = main.steps; }
    if (o->elem) o->elem[idx] = main.e;
    if (o->bary) { o->bary[2 * idx] = main.bary[0]; o->bary[2 * idx + 1] = main.bary[1]; }
    if (o->xbar) for (int i = 0; i < 3; ++i) o->xbar[3 * idx + i] = main.xbar[i];
    if (o->x1) for (int i = 0; i < 3; ++i) o->x1[3 * idx + i] = main.x1[i];
    if (o->x_end) for (int i = 0; i < 3; ++i) o->x_end[3 * idx + i] = main.x_last[i];
    if (mode == 0) return;
    for (int j = 1; j <= s->K; ++j) {
        if (o->kind) o->kind[idx * slots + j] = -1;
        if (o->steps) o->steps[idx * slots + j] = 0;
    }
    if (o->udot) for (int j = 0; j < P; ++j) o->udot[idx * P + j] = 0;
    if (o->dudn) o->dudn[idx] = 0;
    if (o->u_off) o->u_off[idx] = 0;
    if (o->u_plain) o->u_plain[idx] = 0;
    if (o->disp_n) o->disp_n[idx] = 0;
    if (o->disp_t) o->disp_t[idx] = 0;
    if (o->normal) for (int i = 0; i < 3; ++i) o->normal[3 * idx + i] = 0;
    if (main.kind == KIND_ROULETTE) return;   /* Algorithm 2: roulette returns 0 */

    /* BoundaryNormal, oriented away from the walk point */
    double n[3];
    element_normal(s, main.e, n);
    double side = 0;
    for (int i = 0; i < s->dim; ++i) side += n[i] * (main.xbar[i] - main.x_last[i]);
    if (side < 0) for (int i = 0; i < 3; ++i) n[i] = -n[i];

    /* offset point and nested forward walks */
    double xoff[3] = {0, 0, 0};
    for (int i = 0; i < s->dim; ++i) xoff[i] = main.xbar[i] - s->h * n[i];
    if (s->neumann) {   /* mirrored across the Neumann part where the offset crosses it */
        double back[3] = {-n[0], -n[1], -n[2]};
        int he;
        const double th = ray_neumann(s, main.xbar, back, s->h, -1, NULL, -1, NULL, 0.0, &he);
        if (he >= 0) {
            double m[3];
            element_normal(s, he, m);
            double c[3], r[3], rm = 0;
            for (int i = 0; i < 3; ++i) { c[i] = main.xbar[i] + th * back[i]; r[i] = xoff[i] - c[i]; rm += r[i] * m[i]; }
            for (int i = 0; i < s->dim; ++i) xoff[i] = c[i] + r[i] - 2 * rm * m[i];
        }
    }
    /* the nested walks start on the Neumann side(s) the main walk ended on where
     * the offset point lies on it (within 1e-4 eps of its plane) */
    StarStart nst;
    if (s->neumann) {
        double r[3] = {0, 0, 0};
        for (int i = 0; i < s->dim; ++i) r[i] = xoff[i] - main.x_last[i];
        const double on_line = 1e-4 * s->eps;
        const bool k1 = main.on >= 0 && std::fabs(dot3(r, main.n_on)) <= on_line;
        const bool k2 = main.on2 >= 0 && std::fabs(dot3(r, main.n2)) <= on_line;
        if (k1) {
            nst.on = main.on;
            for (int i = 0; i < 3; ++i) nst.n_on[i] = main.n_on[i];
            if (k2) { nst.on2 = main.on2; for (int i = 0; i < 3; ++i) nst.n2[i] = main.n2[i]; }
        } else if (k2) {
            nst.on = main.on2;
            for (int i = 0; i < 3; ++i) nst.n_on[i] = main.n2[i];
        }
    }
    double sum = 0, sum_plain = 0, sum_dn = 0, sum_dt = 0, sum_ball = 0;
    const double* q_cv = s->cv_elem ? s->cv_elem + 4 * (size_t)main.e : NULL;
    for (int j = 1; j <= s->K; ++j) {
        PhaseResult nr = phase_walk(s, adj, xoff, walk_id, (uint32_t)j, s->dudn_mode == 1 ? n : NULL, &nst);
        /* control variate: (q n + t) . (x_end - x_off) has mean zero */
        double disp = 0, dn = 0, dt = 0;
        for (int i = 0; i < s->dim; ++i) dn += n[i] * (nr.x_last[i] - xoff[i]);
        if (q_cv) {
            for (int i = 0; i < s->dim; ++i) dt += q_cv[1 + i] * (nr.x_last[i] - xoff[i]);
            disp = q_cv[0] * dn + dt;
        }
        sum += nr.u - disp;
        sum_plain += nr.u;
        sum_ball += nr.ball_w * nr.u;
        sum_dn += dn;
        sum_dt += dt;
        if (o->kind) o->kind[idx * slots + j] = nr.kind;
        if (o->steps) o->steps[idx * slots + j] = nr.steps;
    }
    double ubar = sum / s->K;
    double g = dirichlet_value(s, main.e, main.bary, main.xbar);
    double dudn = s->dudn_mode == 1 ? sum_ball / s->K   /* Eq. (dudn_mc_estimate) */
                                    : (g - ubar) / s->h;  /* Eq. (dudn_fd_estimate) */
    if (o->dudn) o->dudn[idx] = dudn;
    if (o->u_off) o->u_off[idx] = ubar;
    if (o->u_plain) o->u_plain[idx] = sum_plain / s->K;
    if (o->disp_n) o->disp_n[idx] = sum_dn / s->K;
    if (o->disp_t) o->disp_t[idx] = sum_dt / s->K;
    if (o->normal) for (int i = 0; i < 3; ++i) o->normal[3 * idx + i] = n[i];

    if (!o->udot || P == 0) return;
    /* V_n and the velocity V at xbar, per parameter (explicit surface, Sec. 3.1.2) */
    double w[3];
    vertex_weights(s->dim, main.bary, w);
    const int* el = s->elem + (size_t)s->dim * main.e;
    double gradg[3] = {0, 0, 0};
    double dgdn = 0;
    if (s->data_kind == 1) {
        field_value(s, main.xbar, gradg);
        for (int i = 0; i < s->dim; ++i) dgdn += n[i] * gradg[i];
    } else {
        surface_gradient(s, main.e, gradg);
    }
    for (int j = 0; j < P; ++j) {
        double V[3] = {0, 0, 0};
        if (s->jac) {
            for (int a = 0; a < s->dim; ++a) {
                const double* J = s->jac + ((size_t)el[a] * s->dim) * P;
                for (int k = 0; k < s->dim; ++k) V[k] += w[a] * J[(size_t)k * P + j];
            }
        }
        double Vn = 0;
        for (int k = 0; k < s->dim; ++k) Vn += n[k] * V[k];
        double gdot;
        if (s->data_kind == 1) {
            /* Eq. (boundary_deriv_restricted) with a parameter-free field */
            gdot = dgdn * Vn;
        } else {
            /* Eq. (boundary_deriv_mapped) with dg/dn = 0 */
            double gt = 0;
            if (s->dg_vert)
                for (int a = 0; a < s->dim; ++a) gt += w[a] * s->dg_vert[(size_t)el[a] * P + j];
            double tang = 0;
            for (int k = 0; k < s->dim; ++k) tang += gradg[k] * V[k];
            gdot = gt - tang;
        }
        /* Eq. (wos_deriv), shell case */
        o->udot[idx * P + j] = gdot - Vn * dudn;
    }
}

/* Runs walks_per_point walks from each query point.  Walk (p, w) has global
 * id walk_id_base + p * walks_per_point + w and writes output row
 * p * walks_per_point + w.  mode 0: Algorithm 1 only; mode 1: Algorithm 2. */
int oracle_run_walks(const oracle_scene* s, int n_query, const double* xq, int walks_per_point,
                     uint64_t walk_id_base, int mode, int n_threads, const oracle_walk_out* o) {
    if (!s || !xq || !o || n_query < 0 || walks_per_point < 0) return 1;
    if (s->dim != 2 && s->dim != 3) return 1;
    if (mode == 1 && s->K < 1) return 1;
    if (s->neumann && s->dudn_mode != 0) return 1;   /* the ball-gradient estimator needs a ball in the domain */
    const Adjacency adj = build_adjacency(s);
    long long total = (long long)n_query * walks_per_point;
#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
#endif
    for (long long i = 0; i < total; ++i) {
        long long p = i / walks_per_point;
        run_one(s, &adj, xq + (size_t)p * s->dim, walk_id_base + (uint64_t)i, mode, o, (size_t)i);
    }
    (void)n_threads;
    return 0;
}

/* Inside test by ray parity: count crossings of the ray x + t dir (t > 0)
 * with every element; odd means inside the region the boundary encloses. */
int oracle_inside(const oracle_scene* s, int n, const double* xq, int* inside) {
    const double d2[2] = {0.6180339887498949, 0.7861513777574233};
    const double d3[3] = {0.5773502691896258 * 0.9, 0.5773502691896258 * 1.1, 0.0};
    double dir3[3] = {d3[0], d3[1], std::sqrt(1 - d3[0] * d3[0] - d3[1] * d3[1])};
    for (int i = 0; i < n; ++i) {
        const double* p = xq + (size_t)i * s->dim;
        int count = 0;
        for (int e = 0; e < s->n_elem; ++e) {
            if (s->dim == 2) {
                const int* el = s->elem + 2 * e;
                const double* a = s->vert + 2 * el[0];
                const double* b = s->vert + 2 * el[1];
                /* solve p + t d = a + u (b - a) */
                double ex = b[0] - a[0], ey = b[1] - a[1];
                double det = -d2[0] * ey + d2[1] * ex;
                if (det == 0) continue;
                double rx = a[0] - p[0], ry = a[1] - p[1];
                double t = (-rx * ey + ry * ex) / det;
                double u = (d2[0] * ry - d2[1] * rx) / det;
                if (t > 0 && u >= 0 && u < 1) ++count;
            } else {
                const int* el = s->elem + 3 * e;
                const double* a = s->vert + 3 * el[0];
                const double* b = s->vert + 3 * el[1];
                const double* c = s->vert + 3 * el[2];
                double e1[3], e2[3], tv[3];
                for (int k = 0; k < 3; ++k) { e1[k] = b[k] - a[k]; e2[k] = c[k] - a[k]; tv[k] = p[k] - a[k]; }
                double pv[3] = {dir3[1] * e2[2] - dir3[2] * e2[1], dir3[2] * e2[0] - dir3[0] * e2[2],
                                dir3[0] * e2[1] - dir3[1] * e2[0]};
                double det = dot3(e1, pv);
                if (det == 0) continue;
                double u = dot3(tv, pv) / det;
                if (u < 0 || u > 1) continue;
                double qv[3] = {tv[1] * e1[2] - tv[2] * e1[1], tv[2] * e1[0] - tv[0] * e1[2],
                                tv[0] * e1[1] - tv[1] * e1[0]};
                double v = dot3(dir3, qv) / det;
                if (v < 0 || u + v > 1) continue;
                double t = dot3(e2, qv) / det;
                if (t > 0) ++count;
            }
        }
        inside[i] = count & 1;
    }
    return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  /* extern "C" */
