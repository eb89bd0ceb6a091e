// Device helpers of the walk-on-stars step (Sec. 3.4: mixed Dirichlet /
// reflecting Neumann boundaries; the walk-on-stars estimator of Sawhney et
// al. 2023).  From x the walk uses the star-shaped region St(x, R): the points
// of the ball B(x, R) that x sees without crossing the Neumann part, with
// R = max(min(distance to the Dirichlet part - c, distance to the closest
// silhouette point of the Neumann part), eps - c), c = 1e-3 eps the Dirichlet
// clearance.  A step samples a direction (turned into the domain when x lies
// on the Neumann part: turn_inward),
// casts the ray to the first Neumann crossing within R and moves there or to
// x + R v; its survival weight is |S| t^(d-1) |G_R'(t)| for the step length t.
#pragma once
#include "dwos_device.cuh"
#include "dwos_internal.h"

namespace dwos {

// Leaves of a binary BVH in near-first order with pruning: key(lo, hi, child)
// is a lower bound of what any leaf under the child (>= 0 an internal node,
// < 0 ~leaf) with that box can give and leaf(l) may lower `best`; a box whose
// key exceeds best is skipped.  The outsized leaves after
// the tree's are offered first.  Stackless: the walk back up refetches each
// parent and re-orders its children by the same keys.  Returns false if the
// node budget ran out.
template <int DIM, class Key, class Leaf>
__device__ __forceinline__ bool bvh_best_first(const float4* __restrict__ nodes, int n_internal, int n_tree, int n_big,
                                               const float& best, Key key, Leaf leaf) {
    for (int p = n_tree; p < n_tree + n_big; ++p) leaf(p);
    if (n_tree == 0) return true;
    if (n_internal == 0) { leaf(0); return true; }
    int budget = 4 * n_internal + 64;
    int node = 0, from = kFromParent;
    for (;;) {
        if (--budget < 0) return false;
        float lo0[DIM], hi0[DIM], lo1[DIM], hi1[DIM];
        int c0, c1, parent;
        load_node<DIM>(nodes, node, lo0, hi0, lo1, hi1, c0, c1, parent);
        const float k0 = c0 == kEmptyChild ? kInf : key(lo0, hi0, c0);
        const float k1 = c1 == kEmptyChild ? kInf : key(lo1, hi1, c1);
        const bool first0 = k0 <= k1;
        const int nearc = first0 ? c0 : c1, farc = first0 ? c1 : c0;
        const float kn = first0 ? k0 : k1, kf = first0 ? k1 : k0;
        int state = (from == kFromParent) ? 0 : (from == nearc ? 1 : 2);
        int next = kFromParent;
        for (;;) {
            int cand = kFromParent;
            if (state == 0) { if (kn <= best) cand = nearc; else state = 2; }
            if (state == 1) { if (kf <= best) cand = farc; }
            if (cand == kFromParent || cand == kEmptyChild) break;
            if (cand < 0) {
                leaf(~cand);
                state = (state == 0) ? 1 : 2;
                continue;
            }
            next = cand;
            break;
        }
        if (next != kFromParent) { from = kFromParent; node = next; continue; }
        if (node == 0) return true;
        from = node;
        node = parent;
    }
}

template <int DIM>
__device__ __forceinline__ void vload(const float* __restrict__ vert, int v, float* out) {
#pragma unroll
    for (int k = 0; k < DIM; ++k) out[k] = __ldg(vert + (size_t)DIM * v + k);
}

// The silhouette rule from the two side tests s1, s2 and their scales m1, m2
// (the products of the lengths involved): a side test within a relative 1e-4
// of zero counts as collinear / coplanar.  Both collinear: the boundary runs
// straight on through the vertex (flat across the edge) as seen from x, no
// silhouette; one collinear and the other turning away: a silhouette; else a
// silhouette when both neighbours lie on the same side.
__device__ __forceinline__ bool silhouette_rule(float s1, float m1, float s2, float m2) {
    const bool c1 = fabsf(s1) <= 1e-4f * m1, c2 = fabsf(s2) <= 1e-4f * m2;
    if (c1 && c2) return false;
    if (c1 || c2) return true;
    return s1 * s2 > 0.0f;
}

// True where the Neumann part runs straight on through a site, which is then
// a silhouette from no x: at a vertex v between segments vw and vz the unit
// directions w -> v and v -> z agree within a relative 1e-6 (2D, u1 = v - w,
// u2 = z - v); across an edge ab between triangles abc and abz the unit
// normals (b - a) x (c - a) and (z - a) x (b - a) agree within 1e-6 (3D).
__device__ __forceinline__ bool runs_straight_on(const float* u1, const float* u2) {
    const float dot = u1[0] * u2[0] + u1[1] * u2[1] + u1[2] * u2[2];
    const float n1 = u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2];
    const float n2 = u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2];
    return dot >= (1.0f - 1e-6f) * sqrtf(n1 * n2);
}

// True if Neumann element f (-1: none) has exactly the vertices p, q (and r
// in 3D).
template <int DIM>
__device__ __forceinline__ bool element_is(const DevNeumann& N, int f, int p, int q, int r) {
    if (f < 0) return false;
    bool all = true;
    const int want[3] = {p, q, r};
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        bool found = false;
#pragma unroll
        for (int k = 0; k < DIM; ++k) found = found || __ldg(N.elem + (size_t)DIM * f + k) == want[i];
        all = all && found;
    }
    return all;
}

// True if the box (lo, hi) of the silhouette tree's child (>= 0 an internal
// node, < 0 ~leaf) holds no silhouette point seen from x: its normal cone
// shows that every normal of its sites has one sign against every direction
// from the box to x, with room to spare for the silhouette rule's collinear
// tolerance: |phi - pi/2| > theta + beta + m (phi: cone axis to the box
// centre's direction, beta: the box's angular radius seen from x; m = 1.1 tau
// + 2e-3 rad for FP32 rounding, tau the tolerance's angle, cone_tol (d + rho +
// cone_lmax), bounded by 0.5, above which nothing is skipped).
template <int DIM>
__device__ __forceinline__ bool cone_prunes(const DevNeumann& N, const float* x, const float* lo, const float* hi,
                                         int child) {
    const float4 cn = child >= 0 ? __ldg(N.sil_cone_node + child) : __ldg(N.sil_cone_leaf + ~child);
    if (cn.w >= 3.0f) return false;
    const float ax[3] = {cn.x, cn.y, cn.z};
    float r2 = 0.0f, d2 = 0.0f, dot = 0.0f;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        const float hh = 0.5f * (hi[i] - lo[i]), w = x[i] - 0.5f * (lo[i] + hi[i]);
        r2 = fmaf(hh, hh, r2);
        d2 = fmaf(w, w, d2);
        dot = fmaf(ax[i], w, dot);
    }
    if (d2 <= r2) return false;
    const float d = sqrtf(d2), rho = sqrtf(r2);
    const float tau = N.cone_tol * (d + rho + N.cone_lmax);
    if (tau >= 0.5f) return false;
    const float beta = asinf(fminf(rho / d, 1.0f));
    const float phi = acosf(fminf(fmaxf(dot / d, -1.0f), 1.0f));
    return fabsf(phi - 1.57079633f) > cn.w + beta + fmaf(1.1f, tau, 2e-3f);
}

// Squared distance from x to the closest silhouette point of the Neumann part
// below `bound2` (bound2 itself if there is none), over the candidate sites
// (DevNeumann::sites): vertices (2D) or edges (3D) where the part ends, or
// whose two elements lie on the same side of the ray (2D) or plane (3D)
// through x (silhouette_rule) without the part running straight on there.
// The walk sits on elements on and on2 (-1: none): a side test whose points
// span one of them is zero by definition (x lies on it).
// CONES: the tree has normal cones (a separate kernel instantiation: the cone
// test's code costs the kernels without cones 4-9 % even where it never runs).
template <int DIM, bool CONES>
__device__ __forceinline__ float silhouette_dist2(const DevNeumann& N, const float* x, float bound2, int on, int on2,
                                                  bool& ok) {
    float best = bound2;
    auto key = [&](const float* lo, const float* hi, int child) {
        const float k = box_dist2<DIM>(x, lo, hi);
        if constexpr (CONES) {
            if (k < best && cone_prunes<DIM>(N, x, lo, hi, child)) return kInf;
        }
        return k;
    };
    auto test = [&](int e, int j) {
        const int* ev = N.elem + (size_t)DIM * e;
        if (DIM == 2) {
            float v[2], w[2];
            const int iv = __ldg(ev + j);
            vload<2>(N.vert, iv, v);
            const float rv0 = v[0] - x[0], rv1 = v[1] - x[1];
            const float d2 = rv0 * rv0 + rv1 * rv1;
            if (d2 >= best) return;
            const int nb = __ldg(N.adj + 2 * (size_t)e + j);
            bool sil = nb < 0;
            if (!sil) {
                float z[2];
                vload<2>(N.vert, __ldg(ev + 1 - j), w);
                vload<2>(N.vert, nb, z);
                const float u1[3] = {v[0] - w[0], v[1] - w[1], 0.0f}, u2[3] = {z[0] - v[0], z[1] - v[1], 0.0f};
                if (runs_straight_on(u1, u2)) return;
                const float rw0 = w[0] - x[0], rw1 = w[1] - x[1], rz0 = z[0] - x[0], rz1 = z[1] - x[1];
                const float lv = sqrtf(d2);
                const bool own1 = e == on || e == on2;
                const bool own2 = element_is<2>(N, on, iv, nb, -1) || element_is<2>(N, on2, iv, nb, -1);
                sil = silhouette_rule(own1 ? 0.0f : rv0 * rw1 - rv1 * rw0, lv * sqrtf(rw0 * rw0 + rw1 * rw1),
                                      own2 ? 0.0f : rv0 * rz1 - rv1 * rz0, lv * sqrtf(rz0 * rz0 + rz1 * rz1));
            }
            if (sil) best = d2;
        } else {
            float a[3], b[3];
            const int ia = __ldg(ev + j), ib = __ldg(ev + (j + 1) % 3);
            vload<3>(N.vert, ia, a);
            vload<3>(N.vert, ib, b);
            const float ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
            const float ra[3] = {a[0] - x[0], a[1] - x[1], a[2] - x[2]};
            const float len2 = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
            float t = len2 > 0.0f ? -(ra[0] * ab[0] + ra[1] * ab[1] + ra[2] * ab[2]) / len2 : 0.0f;
            t = fminf(fmaxf(t, 0.0f), 1.0f);
            const float o[3] = {ra[0] + t * ab[0], ra[1] + t * ab[1], ra[2] + t * ab[2]};
            const float d2 = o[0] * o[0] + o[1] * o[1] + o[2] * o[2];
            if (d2 >= best) return;
            const int nb = __ldg(N.adj + 3 * (size_t)e + j);
            bool sil = nb < 0;
            if (!sil) {
                float c[3], z[3];
                vload<3>(N.vert, __ldg(ev + (j + 2) % 3), c);
                vload<3>(N.vert, nb, z);
                const float ac[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
                const float az[3] = {z[0] - a[0], z[1] - a[1], z[2] - a[2]};
                const float u1[3] = {ab[1] * ac[2] - ab[2] * ac[1], ab[2] * ac[0] - ab[0] * ac[2],
                                     ab[0] * ac[1] - ab[1] * ac[0]};
                const float u2[3] = {az[1] * ab[2] - az[2] * ab[1], az[2] * ab[0] - az[0] * ab[2],
                                     az[0] * ab[1] - az[1] * ab[0]};
                if (runs_straight_on(u1, u2)) return;
                const float rb[3] = {b[0] - x[0], b[1] - x[1], b[2] - x[2]};
                const float n[3] = {ra[1] * rb[2] - ra[2] * rb[1], ra[2] * rb[0] - ra[0] * rb[2],
                                    ra[0] * rb[1] - ra[1] * rb[0]};
                const float rc[3] = {c[0] - x[0], c[1] - x[1], c[2] - x[2]};
                const float rz[3] = {z[0] - x[0], z[1] - x[1], z[2] - x[2]};
                const float ln = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
                const bool own1 = e == on || e == on2;
                const bool own2 = element_is<3>(N, on, ia, ib, nb) || element_is<3>(N, on2, ia, ib, nb);
                sil = silhouette_rule(own1 ? 0.0f : n[0] * rc[0] + n[1] * rc[1] + n[2] * rc[2],
                                      ln * sqrtf(rc[0] * rc[0] + rc[1] * rc[1] + rc[2] * rc[2]),
                                      own2 ? 0.0f : n[0] * rz[0] + n[1] * rz[1] + n[2] * rz[2],
                                      ln * sqrtf(rz[0] * rz[0] + rz[1] * rz[1] + rz[2] * rz[2]));
            }
            if (sil) best = d2;
        }
    };
    // a leaf is a Neumann element with a mask of its candidate endpoints / edges
    auto leaf = [&](int l) {
        const int site = __ldg(N.sites + __ldg(N.sil_prim + l));
#pragma unroll
        for (int j = 0; j < DIM; ++j)
            if ((site >> j) & 1) test(site >> 3, j);
    };
    ok = bvh_best_first<DIM>(N.sil_nodes, N.sil_n_internal, N.sil_n_tree, N.sil_n_big, best, key, leaf);
    return best;
}

// Entry distance of the ray x + t v, t >= 0, into a box (kInf if it misses).
template <int DIM>
__device__ __forceinline__ float ray_box_entry(const float* x, const float* inv, const float* lo, const float* hi) {
    float t0 = 0.0f, t1 = kInf;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const float a = (lo[k] - x[k]) * inv[k], b = (hi[k] - x[k]) * inv[k];
        t0 = fmaxf(t0, fminf(a, b));
        t1 = fminf(t1, fmaxf(a, b));
    }
    return t0 <= t1 ? t0 : kInf;
}

// Unit normal (up to orientation) of Neumann element e.
template <int DIM>
__device__ __forceinline__ void neumann_normal(const DevNeumann& N, int e, float* m) {
    const int* ev = N.elem + (size_t)DIM * e;
    float a[DIM], b[DIM];
    vload<DIM>(N.vert, __ldg(ev), a);
    vload<DIM>(N.vert, __ldg(ev + 1), b);
    if (DIM == 2) {
        m[0] = b[1] - a[1];
        m[1] = a[0] - b[0];
    } else {
        float c[DIM];
        vload<DIM>(N.vert, __ldg(ev + 2), c);
        const float e1[3] = {b[0] - a[0], b[1] - a[1], b[DIM - 1] - a[DIM - 1]};
        const float e2[3] = {c[0] - a[0], c[1] - a[1], c[DIM - 1] - a[DIM - 1]};
        m[0] = e1[1] * e2[2] - e1[2] * e2[1];
        m[1] = e1[2] * e2[0] - e1[0] * e2[2];
        m[DIM - 1] = e1[0] * e2[1] - e1[1] * e2[0];
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) s = fmaf(m[k], m[k], s);
    s = rsqrtf(s);
#pragma unroll
    for (int k = 0; k < DIM; ++k) m[k] *= s;
}

// True if Neumann element f (compact numbering) lies behind side e (ne: e's
// unit normal, out of the domain): f shares a vertex with e and none of its
// vertices p lies in front of e's line (plane) by more than a relative 1e-6,
// (p - a) . ne >= -1e-6 |p - a| with a e's first vertex.  Flat continuations
// of e and the far side of a reflex corner are behind e: a ray from e into
// the domain cannot reach them.
template <int DIM>
__device__ __forceinline__ bool behind_side(const DevNeumann& N, int e, const float* ne, int f) {
    int ev[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) ev[j] = __ldg(N.elem + (size_t)DIM * e + j);
    bool shared = false;
    int fv[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        fv[k] = __ldg(N.elem + (size_t)DIM * f + k);
#pragma unroll
        for (int j = 0; j < DIM; ++j) shared = shared || fv[k] == ev[j];
    }
    if (!shared) return false;
    float a[DIM];
    vload<DIM>(N.vert, ev[0], a);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        float p[DIM], dn = 0.0f, r2 = 0.0f;
        vload<DIM>(N.vert, fv[k], p);
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            const float r = p[i] - a[i];
            dn = fmaf(r, ne[i], dn);
            r2 = fmaf(r, r, r2);
        }
        if (dn < -1e-6f * sqrtf(r2)) return false;
    }
    return true;
}

// True if Neumann element f lies on the line (plane) of side e through x
// (ne: e's unit normal): their normals are parallel within a relative 1e-6
// and f's line (plane) passes within on_line of x.  A ray from x does not
// cross it, whatever rounding makes of t (a direction nearly along the line
// meets f's line at an arbitrary t).
template <int DIM>
__device__ __forceinline__ bool coplanar_side(const DevNeumann& N, const float* x, const float* ne, int f,
                                              float on_line) {
    float m[3] = {0.0f, 0.0f, 0.0f};
    neumann_normal<DIM>(N, f, m);
    float c = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) c = fmaf(m[k], ne[k], c);
    if (fabsf(c) < 1.0f - 1e-6f) return false;
    float a[DIM], r = 0.0f;
    vload<DIM>(N.vert, __ldg(N.elem + (size_t)DIM * f), a);
#pragma unroll
    for (int k = 0; k < DIM; ++k) r = fmaf(x[k] - a[k], m[k], r);
    return fabsf(r) <= on_line;
}

// The side tests out of line: in 3D the walk-on-stars kernel's code outgrows
// the instruction cache, and these run only for a candidate hit while the
// walk sits on a side (3D walk kernel 6 % faster; in 2D inline is 5-7 %
// faster).
template <int DIM>
__device__ __noinline__ bool behind_side_ool(const DevNeumann& N, int e, const float* ne, int f) {
    return behind_side<DIM>(N, e, ne, f);
}
template <int DIM>
__device__ __noinline__ bool coplanar_side_ool(const DevNeumann& N, const float* x, const float* ne, int f,
                                               float on_line) {
    return coplanar_side<DIM>(N, x, ne, f, on_line);
}
template <int DIM>
__device__ __forceinline__ bool skipped_from_side(const DevNeumann& N, const float* x, int e, const float* ne, int f,
                                                  float on_line) {
    if constexpr (DIM == 3)
        return behind_side_ool<3>(N, e, ne, f) || coplanar_side_ool<3>(N, x, ne, f, on_line);
    else
        return behind_side<DIM>(N, e, ne, f) || coplanar_side<DIM>(N, x, ne, f, on_line);
}

// First crossing of the ray x + t v (0 < t < tmax) with a Neumann element
// other than `skip` and `skip2` (compact numbering; the sides the walk sits
// on, -1 for none, with their unit normals n_skip, n_skip2 out of the domain),
// the elements behind them (behind_side) and those on their lines (planes)
// through x (coplanar_side): returns t (tmax if none) and the element in hit
// (-1 if none).  A crossing up to a relative 1e-5 plus
// on_line beyond tmax counts, at tmax: where the sphere of radius tmax meets
// the Neumann part, a direction that ends there lands on the boundary, and
// rounding (of the landing point too: a relative tolerance alone is below it
// for short rays) must not leave the walk unaware of it.
template <int DIM>
__device__ __forceinline__ float ray_neumann(const DevNeumann& N, const float* x, const float* v, float tmax, int skip,
                                             const float* n_skip, int skip2, const float* n_skip2, float on_line,
                                             int& hit, bool& ok) {
    float best = fmaf(tmax, 1e-5f, tmax) + on_line;
    hit = -1;
    float inv[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) inv[k] = 1.0f / v[k];
    auto key = [&](const float* lo, const float* hi, int) { return ray_box_entry<DIM>(x, inv, lo, hi); };
    auto leaf = [&](int l) {
        const int e = __ldg(N.prim_elem + l);
        if (e == skip || e == skip2) return;
        float t;
        if (DIM == 2) {
            const float4 s = __ldg(N.prims + l);
            const float ab0 = s.z - s.x, ab1 = s.w - s.y, ax0 = s.x - x[0], ax1 = s.y - x[1];
            const float den = v[0] * ab1 - v[1] * ab0;
            if (den == 0.0f) return;
            t = (ax0 * ab1 - ax1 * ab0) / den;
            const float u = (ax0 * v[1] - ax1 * v[0]) / den;
            if (!(u >= -1e-5f && u <= 1.0f + 1e-5f)) return;     // no ray slips between two neighbours
        } else {
            const float4 a = __ldg(N.prims + 3 * l), b = __ldg(N.prims + 3 * l + 1), c = __ldg(N.prims + 3 * l + 2);
            const float e1[3] = {b.x - a.x, b.y - a.y, b.z - a.z}, e2[3] = {c.x - a.x, c.y - a.y, c.z - a.z};
            const float tv[3] = {x[0] - a.x, x[1] - a.y, x[2] - a.z};
            const float p[3] = {v[1] * e2[2] - v[2] * e2[1], v[2] * e2[0] - v[0] * e2[2], v[0] * e2[1] - v[1] * e2[0]};
            const float det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
            if (det == 0.0f) return;
            const float id = 1.0f / det;
            const float u = (tv[0] * p[0] + tv[1] * p[1] + tv[2] * p[2]) * id;
            if (!(u >= -1e-5f && u <= 1.0f + 1e-5f)) return;    // no ray slips between two neighbours
            const float q[3] = {tv[1] * e1[2] - tv[2] * e1[1], tv[2] * e1[0] - tv[0] * e1[2], tv[0] * e1[1] - tv[1] * e1[0]};
            const float w = (v[0] * q[0] + v[1] * q[1] + v[2] * q[2]) * id;
            if (!(w >= -1e-5f && u + w <= 1.0f + 1e-5f)) return;
            t = (e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]) * id;
        }
        if (!(t > 0.0f && t < best)) return;
        if (skip >= 0 && skipped_from_side<DIM>(N, x, skip, n_skip, e, on_line)) return;
        if (skip2 >= 0 && skipped_from_side<DIM>(N, x, skip2, n_skip2, e, on_line)) return;
        best = t;
        hit = e;
    };
    ok = bvh_best_first<DIM>(N.nodes, N.n_internal, N.n_tree, N.n_big, best, key, leaf);
    return fminf(best, tmax);
}


// A direction drawn at a point of the Neumann part, turned into the domain:
// into the inner half-space of the side the walk sits on (n_on, out of the
// domain) by v -> -v; at an edge (corner in 2D), where the walk also lies on
// a second side (n2), by mirrors across the plane it still points out of,
// alternately, at most 4 (a ray in a wedge of interior angle a turns inward
// after at most ceil(pi / a) mirrors: any edge of 45 degrees or more).  At a
// right-angled edge the direction is then uniform over the quarter-space.
template <int DIM>
__device__ __forceinline__ void turn_inward(float* v, int on, const float* n_on, int on2, const float* n2) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) s = fmaf(v[k], n_on[k], s);
    if (on >= 0 && s > 0.0f) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) v[k] = -v[k];
    }
    if (on2 < 0) return;
    for (int m = 0; m < 4; ++m) {
        float a = 0.0f, b = 0.0f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) { a = fmaf(v[k], n2[k], a); b = fmaf(v[k], n_on[k], b); }
        const bool out2 = a > 0.0f;
        if (!out2 && !(b > 0.0f)) return;
        const float c = 2.0f * (out2 ? a : b);
#pragma unroll
        for (int k = 0; k < DIM; ++k) v[k] = fmaf(-c, out2 ? n2[k] : n_on[k], v[k]);
    }
}

// Survival weight of a star step of length t in the ball of radius R:
// |S^(d-1)| t^(d-1) |G_R'(t)|, which is 1 for sigma = 0 and alpha(R) at t = R.
//   2D: kt K1(kt) + kt I1(kt) K0(kR) / I0(kR)
//   3D: (kt cosh(k(R - t)) + sinh(k(R - t))) / sinh(kR)
//     = e^{-kt} (kt (1 + e^{-2a}) - expm1(-2a)) / -expm1(-2kR),  a = k (R - t)
template <int DIM>
__device__ __forceinline__ float star_weight(float k, float t, float R) {
    if (k == 0.0f) return 1.0f;
    if (t >= R) return recursive_weight<DIM>(k, R);
    const float kt = k * t, kR = k * R;
    if (DIM == 2) {
        float w = kt * bessel_k1(kt);
        if (kR < 80.0f) w += kt * cyl_bessel_i1f(kt) * bessel_k0(kR) / cyl_bessel_i0f(kR);
        return w;
    }
    const float a = k * (R - t);
    return expf(-kt) * (kt * (1.0f + expf(-2.0f * a)) - expm1f(-2.0f * a)) / -expm1f(-2.0f * kR);
}

// The Neumann-data term of a walk-on-stars step (Sec. 3.4, Eq. mixed_bvp with
// Robin coefficient 0 and data h = du/dn, n out of the domain).  Green's second
// identity on the star St(x, R) adds (1 / a(x)) times the integral of
// G_R(x, z) h(z) over the part of the Neumann boundary in the ball that x sees,
// a(x) the share of the directions around x that point into the domain (1
// inside, 1/2 on a side, (pi - the angle between the two normals) / 2 pi at an
// edge).  One sample: the Neumann elements closer to x than R (1 - 1e-4) and
// not wholly behind a side the walk sits on (every vertex more than 2e-4 eps
// behind its plane through x: no point of them is seen) are the candidates, of total measure A (length in 2D, area in 3D; the margin
// leaves out the elements that only touch the ball at a silhouette point,
// whose distance is R itself, and parts within 1e-4 R of the sphere, where G_R
// is below 1e-4 of its size); one is drawn with
// probability proportional to its measure as the candidate with the least
// -log(U_c) / |e_c| (the draw does not depend on the order in which the tree
// offers them), U_c = fmix32(w + (c + 1) 0x9E3779B9) as a uniform, w word 2 of
// block 2 of the step, c the compact element, fmix32 the 32-bit finaliser of
// Appleby's MurmurHash3 (a bijection: each U_c is uniform over w); z uniform on
// it (block 2, words 0 and 1).  The sample
// is A G_R(|z - x|) h / a(x) if |z - x| < R and x sees z, else 0.  x sees z if z
// lies on a side the walk sits on; else if z is not behind those sides (an
// element behind a side by the ray rule, or a point (z - x) . n > on_line out
// of its plane, unless the element lies on the side's plane) and no Neumann
// element crosses the segment before 1 - 1e-4 of its length.  Out of line:
// only a walk over a boundary with Neumann data runs it.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

struct Vec3 { float v[3]; };
struct DataSample { float w; int ok; };

template <int DIM>
__device__ __noinline__ DataSample neumann_data_sample(const DevNeumann& N, Vec3 xp, float R, int on, Vec3 non,
                                                       int on2, Vec3 nn2, float on_line, float k, uint32_t seed_lo,
                                                       uint32_t seed_hi, unsigned long long wid, uint32_t step,
                                                       uint32_t phase) {
    const float* x = xp.v;
    const float R2 = R * R, C2 = R2 * (1.0f - 2e-4f), behind_tol = 2.0f * on_line;
    float A = 0.0f, best_key = kInf;
    int pick = -1;
    const U4 r = draw_block(seed_lo, seed_hi, wid, step, phase, 2u);
    auto key = [&](const float* lo, const float* hi, int) { return box_dist2<DIM>(x, lo, hi); };
    auto leaf = [&](int l) {
        if (!(prim_dist2<DIM>(N.prims, l, x) < C2)) return;
        float m;
        if (DIM == 2) {
            const float4 s = __ldg(N.prims + l);
            for (int j = 0; j < 2; ++j) {
                if ((j ? on2 : on) < 0) continue;
                const float* n = j ? nn2.v : non.v;
                if (fmaf(s.x - x[0], n[0], (s.y - x[1]) * n[1]) > behind_tol &&
                    fmaf(s.z - x[0], n[0], (s.w - x[1]) * n[1]) > behind_tol) return;
            }
            m = sqrtf((s.z - s.x) * (s.z - s.x) + (s.w - s.y) * (s.w - s.y));
        } else {
            const float4 a = __ldg(N.prims + 3 * l), b = __ldg(N.prims + 3 * l + 1), c = __ldg(N.prims + 3 * l + 2);
            for (int j = 0; j < 2; ++j) {
                if ((j ? on2 : on) < 0) continue;
                const float* n = j ? nn2.v : non.v;
                auto ahead = [&](float4 p) {
                    return fmaf(p.x - x[0], n[0], fmaf(p.y - x[1], n[1], (p.z - x[DIM - 1]) * n[DIM - 1]));
                };
                if (ahead(a) > behind_tol && ahead(b) > behind_tol && ahead(c) > behind_tol) return;
            }
            const float e1[3] = {b.x - a.x, b.y - a.y, b.z - a.z}, e2[3] = {c.x - a.x, c.y - a.y, c.z - a.z};
            const float w0 = e1[1] * e2[2] - e1[2] * e2[1], w1 = e1[2] * e2[0] - e1[0] * e2[2];
            const float w2 = e1[0] * e2[1] - e1[1] * e2[0];
            m = 0.5f * sqrtf(w0 * w0 + w1 * w1 + w2 * w2);
        }
        if (!(m > 0.0f)) return;
        A += m;
        const int e = __ldg(N.prim_elem + l);
        const float kc = -logf(u01(fmix32(r.z + (uint32_t)(e + 1) * 0x9E3779B9u))) / m;
        if (kc < best_key) { best_key = kc; pick = l; }
    };
    DataSample out{0.0f, 1};
    out.ok = bvh_best_first<DIM>(N.nodes, N.n_internal, N.n_tree, N.n_big, C2, key, leaf) ? 1 : 0;
    if (pick < 0) return out;
    const float u0 = u01(r.x), u1 = u01(r.y);
    float z[DIM];
    if (DIM == 2) {
        const float4 s = __ldg(N.prims + pick);
        z[0] = fmaf(u0, s.z - s.x, s.x);
        z[1] = fmaf(u0, s.w - s.y, s.y);
    } else {
        const float4 a = __ldg(N.prims + 3 * pick), b = __ldg(N.prims + 3 * pick + 1), c = __ldg(N.prims + 3 * pick + 2);
        const float q = sqrtf(u0), wb = q * (1.0f - u1), wc = q * u1, wa = 1.0f - q;
        z[0] = wa * a.x + wb * b.x + wc * c.x;
        z[1] = wa * a.y + wb * b.y + wc * c.y;
        z[DIM - 1] = wa * a.z + wb * b.z + wc * c.z;
    }
    float v[3] = {0.0f, 0.0f, 0.0f}, t2 = 0.0f;
#pragma unroll
    for (int i = 0; i < DIM; ++i) { v[i] = z[i] - x[i]; t2 = fmaf(v[i], v[i], t2); }
    const float t = sqrtf(t2);
    if (!(t < R) || !(t > 0.0f)) return out;
    const int pe = __ldg(N.prim_elem + pick);
    if (pe != on && pe != on2) {
        const int side[2] = {on, on2};
        const float* nrm[2] = {non.v, nn2.v};
        for (int j = 0; j < 2; ++j) {
            if (side[j] < 0) continue;
            if (coplanar_side<DIM>(N, x, nrm[j], pe, on_line)) continue;
            float dn = 0.0f;
#pragma unroll
            for (int i = 0; i < DIM; ++i) dn = fmaf(v[i], nrm[j][i], dn);
            if (dn > on_line || behind_side<DIM>(N, side[j], nrm[j], pe)) return out;
        }
        const float it = 1.0f / t;
#pragma unroll
        for (int i = 0; i < DIM; ++i) v[i] *= it;
        int hit;
        bool ok = true;
        ray_neumann<DIM>(N, x, v, t * (1.0f - 1e-4f), on, non.v, on2, nn2.v, 0.0f, hit, ok);
        if (!ok) out.ok = 0;
        if (hit >= 0) return out;
    }
    float share = 1.0f;
    if (on2 >= 0) {
        float c = 0.0f;
#pragma unroll
        for (int i = 0; i < DIM; ++i) c = fmaf(non.v[i], nn2.v[i], c);
        share = (3.14159265358979f - acosf(fminf(1.0f, fmaxf(-1.0f, c)))) * 0.159154943091895f;
    } else if (on >= 0) {
        share = 0.5f;
    }
    // G_R(t): the source weight of the ball at radius t over the ball's volume
    const float rho = t / R;
    const float uu = DIM == 2 ? rho * rho : rho * rho * rho;
    const float vol = DIM == 2 ? 3.14159265358979f * R2 : 4.18879020478639f * R2 * R;
    out.w = A * (source_weight<DIM>(k, R, uu) / vol) * __ldg(N.flux + pe) / share;
    return out;
}

}  // namespace dwos
