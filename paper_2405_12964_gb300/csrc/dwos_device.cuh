// Device-side building blocks of the walk-on-spheres library (sm_103a).
//
//  - Philox4x32-10 counter RNG (Salmon et al., SC'11) and the uniform map
//  - uniform sphere / ball sampling (Algorithm 1: SampleUnitSphere, SampleUnitBall)
//  - the ball Green's function source weight |B| G and the recursive weight
//    alpha = P |dB| for the screened Poisson equation (Sec. 3.3.1; G and P are
//    derived from the PDE because the paper defers them to WoSt App. A)
//  - closest point on a segment / triangle (DistanceToBoundary, Algorithm 1)
//  - BVH node layout and a stackless, near-child-first closest-point traversal
//    over parent links (Hapala et al. 2011 style state machine)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dwos {

constexpr int kFromParent = 0x7fffffff;   // traversal state: entered from above
constexpr int kEmptyChild = 0x7ffffffe;   // child slot with an empty box
constexpr float kInf = __builtin_inff();

// ---------------------------------------------------------------------------
// Philox4x32-10: ten rounds, two 32x32 multiplies per round, key bumped by the
// Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// ((x >> 9) * 2 + 1) * 2^-24: an odd multiple of 2^-24 in (0, 1), exact in FP32.
__device__ __forceinline__ float u01(uint32_t x) {
    return (float)((x >> 9) * 2u + 1u) * 5.9604644775390625e-8f;
}

// One Philox block of a walk step.  counter = (id lo, id hi, step, phase<<8 | block)
__device__ __forceinline__ U4 draw_block(uint32_t seed_lo, uint32_t seed_hi, unsigned long long walk_id,
                                         uint32_t step, uint32_t phase, uint32_t block) {
    U4 c{(uint32_t)walk_id, (uint32_t)(walk_id >> 32), step, (phase << 8) | block};
    return philox(c, seed_lo, seed_hi);
}

// ---------------------------------------------------------------------------
// Green's function weights on a ball of radius d (k = sqrt(sigma)).
// ---------------------------------------------------------------------------
// Modified Bessel K0 for x > 0: Abramowitz & Stegun 9.8.5 (x <= 2, with I0)
// and 9.8.6 (x > 2) polynomial approximations (|error| < 2e-7 relative).
__device__ __forceinline__ float bessel_k0(float x) {
    if (x <= 2.0f) {
        const float t = 0.25f * x * x;   // (x/2)^2
        float p = 0.74e-5f;
        p = fmaf(p, t, 0.10750e-3f);
        p = fmaf(p, t, 0.262698e-2f);
        p = fmaf(p, t, 0.3488590e-1f);
        p = fmaf(p, t, 0.23069756f);
        p = fmaf(p, t, 0.42278420f);
        p = fmaf(p, t, -0.57721566f);
        return -logf(0.5f * x) * cyl_bessel_i0f(x) + p;
    }
    const float t = 2.0f / x;
    float p = 0.00053208f;
    p = fmaf(p, t, -0.00251540f);
    p = fmaf(p, t, 0.00587872f);
    p = fmaf(p, t, -0.01062446f);
    p = fmaf(p, t, 0.02189568f);
    p = fmaf(p, t, -0.07832358f);
    p = fmaf(p, t, 1.25331414f);
    return expf(-x) * rsqrtf(x) * p;
}

// Modified Bessel K1 for x > 0: Abramowitz & Stegun 9.8.7 (x <= 2, with I1)
// and 9.8.8 (x > 2) polynomial approximations.
__device__ __forceinline__ float bessel_k1(float x) {
    if (x <= 2.0f) {
        const float t = 0.25f * x * x;   // (x/2)^2
        float p = -0.00004686f;
        p = fmaf(p, t, -0.00110404f);
        p = fmaf(p, t, -0.01919402f);
        p = fmaf(p, t, -0.18156897f);
        p = fmaf(p, t, -0.67278579f);
        p = fmaf(p, t, 0.15443144f);
        p = fmaf(p, t, 1.0f);             // x K1(x) = x log(x/2) I1(x) + p
        return logf(0.5f * x) * cyl_bessel_i1f(x) + p / x;
    }
    const float t = 2.0f / x;
    float p = -0.00068245f;
    p = fmaf(p, t, 0.00325614f);
    p = fmaf(p, t, -0.00780353f);
    p = fmaf(p, t, 0.01504268f);
    p = fmaf(p, t, -0.03655620f);
    p = fmaf(p, t, 0.23498619f);
    p = fmaf(p, t, 1.25331414f);
    return expf(-x) * rsqrtf(x) * p;
}

// Russian roulette of Algorithm 1: true when the walk stops (alpha < u).
// alpha >= exp(-(kd)^2/4) >= 1 - (kd)^2/4 in 2D (I0(x) <= exp(x^2/4)) and
// alpha >= 1 - (kd)^2/6 in 3D (sinh(x)/x <= exp(x^2/6)); when u lies below that
// bound by more than the FP32 error of the full evaluation, the walk survives
// and alpha itself is not needed.  Otherwise alpha is evaluated exactly.
template <int DIM>
__device__ __forceinline__ float recursive_weight(float k, float d);

template <int DIM>
__device__ __forceinline__ bool roulette_stops(float k, float d, float u) {
    if (k == 0.0f) return false;                    // alpha = 1 > u for u in (0, 1)
    const float x = k * d;
    const float lb = 1.0f - x * x * (DIM == 2 ? 0.25f : (1.0f / 6.0f)) - 1e-5f;
    if (u < lb) return false;
    return recursive_weight<DIM>(k, d) < u;
}

// alpha(d) = P(d) |dB(d)|: 1/I0(kd) in 2D, kd/sinh(kd) in 3D, 1 when sigma = 0.
template <int DIM>
__device__ __forceinline__ float recursive_weight(float k, float d) {
    if (k == 0.0f) return 1.0f;
    const float kd = k * d;
    if (DIM == 2) return 1.0f / cyl_bessel_i0f(kd);
    // kd / sinh(kd) = -2 kd e^{-kd} / expm1(-2 kd): no overflow, exact limit 1 at 0
    return -2.0f * kd * expf(-kd) / expm1f(-2.0f * kd);
}

// |B(d)| G_d(r) for the ball sample's radius: u is the Philox uniform that
// sets r = d u^(1/DIM).  The source estimate of Algorithm 1 is this times f.
template <int DIM>
__device__ __forceinline__ float source_weight(float k, float d, float u) {
    const float d2 = d * d;
    if (DIM == 2) {
        if (k == 0.0f) return -0.25f * d2 * logf(u);          // (d^2/2) log(d/r)
        const float rho = sqrtf(u);
        const float kd = k * d, kr = kd * rho;
        float g = bessel_k0(kr);
        if (kd < 80.0f) g -= bessel_k0(kd) * cyl_bessel_i0f(kr) / cyl_bessel_i0f(kd);
        return 0.5f * d2 * g;
    }
    const float rho = cbrtf(u);
    if (k == 0.0f) return (d2 * (1.0f / 3.0f)) * (1.0f / rho - 1.0f);
    const float a = k * d * (1.0f - rho), b = k * d;
    // sinh(a)/sinh(b) = e^{a-b} expm1(-2a) / expm1(-2b)
    const float ratio = expf(a - b) * expm1f(-2.0f * a) / expm1f(-2.0f * b);
    return (d2 * (1.0f / 3.0f)) * ratio / rho;
}

// ---------------------------------------------------------------------------
// Closest point on one element.  Segments: clamp the projection parameter.
// Triangles: Voronoi-region classification (Ericson, Real-Time Collision
// Detection, Sec. 5.1.5).  Both return the squared distance and the weights
// of vertices 1 (and 2).  Divisions use the fast path: the closest point is a
// projection, so the squared distance is stationary in the weights there and
// their ulp-level errors only reach d^2 at second order.
// ---------------------------------------------------------------------------
// Every product is rounded explicitly (fmaf, __fmul_rn), so that the compiler
// cannot contract the expressions differently where it inlines them: a leaf's
// distance is then the same bits in every search path, and ties between
// elements (a shared vertex) resolve the same way whichever path found them.
__device__ __forceinline__ float seg_closest(const float* q, float ax, float ay, float bx, float by,
                                             float& t_out) {
    const float ex = bx - ax, ey = by - ay;
    const float px = q[0] - ax, py = q[1] - ay;
    const float len2 = fmaf(ex, ex, __fmul_rn(ey, ey));
    // fast division: the distance is quadratic in t at its minimum, so an
    // ulp-level error in t does not move d^2 beyond rounding
    float t = len2 > 0.0f ? __fdividef(fmaf(px, ex, __fmul_rn(py, ey)), len2) : 0.0f;
    t = fminf(fmaxf(t, 0.0f), 1.0f);
    const float dx = fmaf(-t, ex, px), dy = fmaf(-t, ey, py);
    t_out = t;
    return fmaf(dx, dx, __fmul_rn(dy, dy));
}

__device__ __forceinline__ float dot3_rn(float ax, float ay, float az, float bx, float by, float bz) {
    return fmaf(ax, bx, fmaf(ay, by, __fmul_rn(az, bz)));
}

__device__ __forceinline__ float tri_closest(const float* q, const float3 a, const float3 b, const float3 c,
                                             float& w1, float& w2) {
    const float3 ab = make_float3(b.x - a.x, b.y - a.y, b.z - a.z);
    const float3 ac = make_float3(c.x - a.x, c.y - a.y, c.z - a.z);
    const float3 ap = make_float3(q[0] - a.x, q[1] - a.y, q[2] - a.z);
    const float d1 = dot3_rn(ab.x, ab.y, ab.z, ap.x, ap.y, ap.z);
    const float d2 = dot3_rn(ac.x, ac.y, ac.z, ap.x, ap.y, ap.z);
    const float3 bp = make_float3(q[0] - b.x, q[1] - b.y, q[2] - b.z);
    const float d3 = dot3_rn(ab.x, ab.y, ab.z, bp.x, bp.y, bp.z);
    const float d4 = dot3_rn(ac.x, ac.y, ac.z, bp.x, bp.y, bp.z);
    const float3 cp = make_float3(q[0] - c.x, q[1] - c.y, q[2] - c.z);
    const float d5 = dot3_rn(ab.x, ab.y, ab.z, cp.x, cp.y, cp.z);
    const float d6 = dot3_rn(ac.x, ac.y, ac.z, cp.x, cp.y, cp.z);
    const float vc = fmaf(d1, d4, -__fmul_rn(d3, d2));
    const float vb = fmaf(d5, d2, -__fmul_rn(d1, d6));
    const float va = fmaf(d3, d6, -__fmul_rn(d5, d4));
    float s, t;
    if (d1 <= 0.0f && d2 <= 0.0f) { s = 0.0f; t = 0.0f; }                          // vertex a
    else if (d3 >= 0.0f && d4 <= d3) { s = 1.0f; t = 0.0f; }                        // vertex b
    else if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) { s = __fdividef(d1, d1 - d3); t = 0.0f; }  // edge ab
    else if (d6 >= 0.0f && d5 <= d6) { s = 0.0f; t = 1.0f; }                        // vertex c
    else if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) { s = 0.0f; t = __fdividef(d2, d2 - d6); }  // edge ac
    else if (va <= 0.0f && (d4 - d3) >= 0.0f && (d5 - d6) >= 0.0f) {                // edge bc
        const float u = __fdividef(d4 - d3, (d4 - d3) + (d5 - d6));
        s = 1.0f - u; t = u;
    } else {                                                                          // face
        const float inv = __fdividef(1.0f, va + vb + vc);
        s = __fmul_rn(vb, inv); t = __fmul_rn(vc, inv);
    }
    const float rx = fmaf(-t, ac.x, fmaf(-s, ab.x, ap.x));
    const float ry = fmaf(-t, ac.y, fmaf(-s, ab.y, ap.y));
    const float rz = fmaf(-t, ac.z, fmaf(-s, ab.z, ap.z));
    w1 = s;
    w2 = t;
    return dot3_rn(rx, ry, rz, rx, ry, rz);
}

// ---------------------------------------------------------------------------
// BVH layout.  Internal node i stores both children's boxes (so a parent's
// fetch decides which child to enter), the child codes (>= 0: internal node,
// < 0: ~leaf index, kEmptyChild: nothing) and its parent (-1 at the root).
//   2D node: 3 float4 = 48 B   [L.lo.xy L.hi.xy] [R.lo.xy R.hi.xy] [left right parent -]
//   3D node: 4 float4 = 64 B   [L.lo.xyz L.hi.x] [L.hi.yz R.lo.xy] [R.lo.z R.hi.xyz] [left right parent -]
// Leaves hold one element each, in Morton order:
//   2D prim: 1 float4 [a.xy b.xy];  3D prim: 3 float4 [a.xyz -] [b.xyz -] [c.xyz -]
// ---------------------------------------------------------------------------
template <int DIM> struct BvhLayout;
template <> struct BvhLayout<2> { static constexpr int kNodeF4 = 3; static constexpr int kPrimF4 = 1; };
template <> struct BvhLayout<3> { static constexpr int kNodeF4 = 4; static constexpr int kPrimF4 = 3; };

// Leaves [0, n_tree) are the LBVH's, in Morton order; leaves [n_tree,
// n_tree + n_big) are outsized elements (much larger than the typical one,
// such as an enclosing box) kept out of the tree so that their boxes do not
// inflate every ancestor's: each query tests them first, by brute force.
// For the hint-seeded ascent: each leaf's parent, and each internal node's
// Morton cell (the box of centroids its key prefix admits; every element
// outside the node's subtree has its centroid outside that box) together with
// r_max, the largest distance from an element's box centre to its corners.
struct BvhView {
    const float4* nodes;
    const float4* prims;
    int root;
    int n_internal;   // internal nodes of the tree (0: no tree)
    int n_tree;       // leaves in the tree
    int n_big;        // outsized elements after the tree's leaves
    int climb;        // 1: climb from a tree-leaf hint; 0: always search from the root
    const int* leaf_parent;
    const float* node_cell;   // 2*DIM floats per internal node: lo, hi
    float r_max;
    int budget = 0;           // node fetches allowed per query; 0: 4 x the inner nodes + 64
};

template <int DIM>
__device__ __forceinline__ float box_dist2(const float* q, const float* lo, const float* hi) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const float e = fmaxf(fmaxf(lo[k] - q[k], q[k] - hi[k]), 0.0f);
        s = fmaf(e, e, s);
    }
    return s;
}

template <int DIM>
__device__ __forceinline__ void load_node(const float4* __restrict__ nodes, int i, float* lo0, float* hi0,
                                          float* lo1, float* hi1, int& c0, int& c1, int& parent) {
    if (DIM == 2) {
        const float4 a = __ldg(nodes + 3 * i + 0);
        const float4 b = __ldg(nodes + 3 * i + 1);
        const float4 m = __ldg(nodes + 3 * i + 2);
        lo0[0] = a.x; lo0[1] = a.y; hi0[0] = a.z; hi0[1] = a.w;
        lo1[0] = b.x; lo1[1] = b.y; hi1[0] = b.z; hi1[1] = b.w;
        c0 = __float_as_int(m.x); c1 = __float_as_int(m.y); parent = __float_as_int(m.z);
    } else {
        const float4 a = __ldg(nodes + 4 * i + 0);
        const float4 b = __ldg(nodes + 4 * i + 1);
        const float4 c = __ldg(nodes + 4 * i + 2);
        const float4 m = __ldg(nodes + 4 * i + 3);
        lo0[0] = a.x; lo0[1] = a.y; lo0[2] = a.z; hi0[0] = a.w;
        hi0[1] = b.x; hi0[2] = b.y; lo1[0] = b.z; lo1[1] = b.w;
        lo1[2] = c.x; hi1[0] = c.y; hi1[1] = c.z; hi1[2] = c.w;
        c0 = __float_as_int(m.x); c1 = __float_as_int(m.y); parent = __float_as_int(m.z);
    }
}

template <int DIM>
__device__ __forceinline__ float prim_dist2(const float4* __restrict__ prims, int p, const float* q) {
    if (DIM == 2) {
        const float4 s = __ldg(prims + p);
        float t;
        return seg_closest(q, s.x, s.y, s.z, s.w, t);
    } else {
        const float4 a = __ldg(prims + 3 * p + 0);
        const float4 b = __ldg(prims + 3 * p + 1);
        const float4 c = __ldg(prims + 3 * p + 2);
        float w1, w2;
        return tri_closest(q, make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z),
                           make_float3(c.x, c.y, c.z), w1, w2);
    }
}

// Squared distance from q to the bounding box of leaf p.
template <int DIM>
__device__ __forceinline__ float prim_box_dist2(const float4* __restrict__ prims, int p, const float* q) {
    float lo[DIM], hi[DIM];
    if (DIM == 2) {
        const float4 s = __ldg(prims + p);
        lo[0] = fminf(s.x, s.z); hi[0] = fmaxf(s.x, s.z);
        lo[1] = fminf(s.y, s.w); hi[1] = fmaxf(s.y, s.w);
    } else {
        const float4 a = __ldg(prims + 3 * p), b = __ldg(prims + 3 * p + 1), c = __ldg(prims + 3 * p + 2);
        lo[0] = fminf(a.x, fminf(b.x, c.x)); hi[0] = fmaxf(a.x, fmaxf(b.x, c.x));
        lo[1] = fminf(a.y, fminf(b.y, c.y)); hi[1] = fmaxf(a.y, fmaxf(b.y, c.y));
        lo[DIM - 1] = fminf(a.z, fminf(b.z, c.z)); hi[DIM - 1] = fmaxf(a.z, fmaxf(b.z, c.z));
    }
    return box_dist2<DIM>(q, lo, hi);
}

// Ties between equally distant leaves (a query whose closest point is a vertex
// shared by two elements) go to the lower leaf index, and a box exactly at the
// bound is still searched, so that every search order, seed and schedule picks
// the same element.
__device__ __forceinline__ bool closer(float d, int p, float best2, int best) {
    return d < best2 || (d == best2 && d < kInf && (unsigned)p < (unsigned)best);
}

// A box is searched while its squared distance is within the bound up to a
// relative 1e-5: the computed distance of a box can round above the computed
// distance of an element inside it, and a tied element must not be pruned.
__device__ __forceinline__ bool within(float box_d2, float best2) {
    return box_d2 <= best2 * 1.00001f;
}

// Top-down search of the subtree under internal node `start` for a leaf
// closer than best2: near-child-first descent; on the way back up each parent
// is refetched and its children re-ordered by the same box distances, so no
// stack is needed.  Returns when it climbs back out of `start`.  The budget
// bounds the node fetches (each node is entered at most three times).
template <int DIM>
__device__ __forceinline__ bool search_subtree(const BvhView& bvh, int start, const float* q, float& best2, int& best,
                                               int& budget, unsigned& n_nodes, unsigned& n_prims) {
    int node = start;
    int from = kFromParent;
    for (;;) {
        if (--budget < 0) return false;
        ++n_nodes;
        float lo0[DIM], hi0[DIM], lo1[DIM], hi1[DIM];
        int c0, c1, parent;
        load_node<DIM>(bvh.nodes, node, lo0, hi0, lo1, hi1, c0, c1, parent);
        const float d0 = box_dist2<DIM>(q, lo0, hi0);
        const float d1 = box_dist2<DIM>(q, lo1, hi1);
        const bool first0 = d0 <= d1;
        const int nearc = first0 ? c0 : c1, farc = first0 ? c1 : c0;
        const float dn = first0 ? d0 : d1, df = first0 ? d1 : d0;
        int state = (from == kFromParent) ? 0 : (from == nearc ? 1 : 2);
        int next = kFromParent;
        for (;;) {
            int cand = kFromParent;
            if (state == 0) { if (within(dn, best2)) cand = nearc; else state = 2; }
            if (state == 1) { if (within(df, best2)) cand = farc; }
            if (cand == kFromParent) break;
            if (cand < 0) {                       // leaf: test in place
                const int p = ~cand;
                ++n_prims;
                const float dd = prim_dist2<DIM>(bvh.prims, p, q);
                if (closer(dd, p, best2, best)) { best2 = dd; best = p; }
                state = (state == 0) ? 1 : 2;
                continue;
            }
            next = cand;
            break;
        }
        if (next != kFromParent) { from = kFromParent; node = next; continue; }
        if (node == start) return true;
        from = node;
        node = parent;
    }
}

// Closest leaf to q.  On entry best2 / best hold an upper bound and its leaf
// (the previous step's closest element: any element's distance bounds the
// minimum), or kInf / -1.  Outsized elements are tested first.  With a tree
// leaf as hint the search climbs from that leaf: at each ancestor the sibling
// subtree is searched if its box is within the bound, and the climb stops once
// the ball of radius best + r_max around q lies inside the ancestor's Morton
// cell (no element outside the ancestor's subtree can then be closer).
// Without one it searches the whole tree from the root.  Returns false if the
// fetch budget was exceeded (never in a valid tree).
template <int DIM>
__device__ __forceinline__ bool closest_leaf(const BvhView& bvh, const float* q, float& best2, int& best,
                                             unsigned& n_nodes, unsigned& n_prims) {
    for (int p = bvh.n_tree; p < bvh.n_tree + bvh.n_big; ++p) {
        if (!within(prim_box_dist2<DIM>(bvh.prims, p, q), best2)) continue;   // cannot be closer
        ++n_prims;
        const float dd = prim_dist2<DIM>(bvh.prims, p, q);
        if (closer(dd, p, best2, best)) { best2 = dd; best = p; }
    }
    if (bvh.n_internal == 0) return true;
    int budget = bvh.budget > 0 ? bvh.budget : 4 * bvh.n_internal + 64;
    if (!bvh.climb || best < 0 || best >= bvh.n_tree || !bvh.leaf_parent)
        return search_subtree<DIM>(bvh, bvh.root, q, best2, best, budget, n_nodes, n_prims);
    int child = ~best;
    int node = __ldg(bvh.leaf_parent + best);
    while (node >= 0) {
        if (--budget < 0) return false;
        ++n_nodes;
        float lo0[DIM], hi0[DIM], lo1[DIM], hi1[DIM];
        int c0, c1, parent;
        load_node<DIM>(bvh.nodes, node, lo0, hi0, lo1, hi1, c0, c1, parent);
        const bool from0 = (c0 == child);
        const int sib = from0 ? c1 : c0;
        if (sib != kEmptyChild) {
            const float ds = from0 ? box_dist2<DIM>(q, lo1, hi1) : box_dist2<DIM>(q, lo0, hi0);
            if (within(ds, best2)) {
                if (sib < 0) {
                    ++n_prims;
                    const float dd = prim_dist2<DIM>(bvh.prims, ~sib, q);
                    if (closer(dd, ~sib, best2, best)) { best2 = dd; best = ~sib; }
                } else if (!search_subtree<DIM>(bvh, sib, q, best2, best, budget, n_nodes, n_prims)) {
                    return false;
                }
            }
        }
        // stop when the ball around q, grown by r_max, lies inside this node's Morton cell
        const float r = sqrtf(best2) + bvh.r_max;
        const float* cell = bvh.node_cell + 2 * DIM * node;
        bool inside = true;
#pragma unroll
        for (int k = 0; k < DIM; ++k)
            inside = inside && (q[k] - r >= __ldg(cell + k)) && (q[k] + r <= __ldg(cell + DIM + k));
        if (inside) return true;
        child = node;
        node = parent;
    }
    return true;
}

// Factor of the ball gradient estimator behind Eq. (dudn_mc_estimate): for
// -Lap u + k^2 u = 0 in a ball of radius R about c and y uniform on its
// sphere, grad u(c) = F(R) E[n_y u(y)].  The l = 1 solutions u = I1(kr) cos t
// (2D) and i1(kr) cos t (3D, i1 the modified spherical Bessel function) give
// F = k / I1(kR) and k / i1(kR); both tend to d / R as k -> 0.
template <int DIM>
__device__ __forceinline__ float gradient_factor(float k, float R) {
    const float z = k * R;
    if (DIM == 2) return k > 0.0f ? k / cyl_bessel_i1f(z) : 2.0f / R;
    if (!(k > 0.0f)) return 3.0f / R;
    if (z < 0.5f) {            // i1(z) = z/3 + z^3/30 + z^5/840 + z^7/45360 + ...
        const float z2 = z * z;
        return k / (z * (1.0f / 3.0f + z2 * (1.0f / 30.0f + z2 * (1.0f / 840.0f + z2 * (1.0f / 45360.0f)))));
    }
    if (z < 20.0f) return k * z * z / (z * coshf(z) - sinhf(z));
    return 2.0f * k * z * z * expf(-z) / (z - 1.0f);   // i1(z) = e^z (z - 1) / (2 z^2) + O(e^-z)
}

// ---- 32-wide BVH searched by a whole warp ---------------------------------
// The binary LBVH collapsed five levels at a time: a wide node holds up to 32
// children in SoA order, lo[DIM][32], hi[DIM][32], code[32] (>= 0: wide node,
// < 0: ~leaf, kEmptyChild: unused slot with an empty box) and, for leaf
// children, the element's vertices vtx[DIM * DIM][32] (segment a, b or
// triangle a, b, c), so that lane j of a warp loads slot j of every array with
// one coalesced request per array, and a visit needs one round trip to memory
// whether its children are nodes or elements.
constexpr int kWide = 32;
constexpr int kWideStack = 224;            // stack entries per warp: 31 x wide depth + 1 (checked at build): depth <= 7
constexpr unsigned kWarpAll = 0xffffffffu;
template <int DIM> struct WideLayout {
    static constexpr int kVtx = (2 * DIM + 1) * kWide;              // offset of the vertex arrays
    static constexpr int kFloats = (2 * DIM + 1 + DIM * DIM) * kWide;
};

struct WideView {
    const float* wnodes;   // n_wide nodes of WideLayout<DIM>::kFloats floats, root first
    const float4* prims;
    int n_wide;
    int n_tree;
    int budget = 0;        // wide-node visits allowed per query; 0: the tree's node count
};

// Closest tree leaf for every lane in `need`, one query at a time, with all
// 32 lanes working on it: each lane takes one child slot of the current wide
// node, leaf children are measured exactly in parallel and reduced with
// shuffles (ties to the lower leaf index), and the inner children that can
// still hold a closer leaf go on the warp's stack in shared memory with the
// nearest on top (depth-first, nearest child first, the others in Morton
// order, all pruned by the running bound when popped).  n_nodes counts node
// visits (a leaf child's vertices come with its node).
// best2 / best hold each lane's bound on entry (kInf / -1 without one) and
// the result on exit.  Called by all 32 lanes with the same `need` and each
// lane's own view (lanes may belong to different problems).  Returns error
// bits: 1 if a query popped more nodes than the tree has, 4 if the stack
// would overflow (excluded by the build's depth check).
template <int DIM>
__device__ __forceinline__ int wide_closest(const WideView& mine, unsigned need, const float* q_lane, float& best2,
                                            int& best, float2* stk, unsigned& n_nodes, unsigned& n_prims) {
    const int lane = threadIdx.x & 31;
    int err = 0;
    while (need) {
        const int src = __ffs(need) - 1;
        need &= need - 1;
        float q[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) q[k] = __shfl_sync(kWarpAll, q_lane[k], src);
        float b2 = __shfl_sync(kWarpAll, best2, src);
        int bi = __shfl_sync(kWarpAll, best, src);
        const float* wn = reinterpret_cast<const float*>(
            __shfl_sync(kWarpAll, reinterpret_cast<unsigned long long>(mine.wnodes), src));
        const float4* prims = reinterpret_cast<const float4*>(
            __shfl_sync(kWarpAll, reinterpret_cast<unsigned long long>(mine.prims), src));
        const int n_wide = __shfl_sync(kWarpAll, mine.n_wide, src);
        const int n_tree = __shfl_sync(kWarpAll, mine.n_tree, src);
        const int cap = __shfl_sync(kWarpAll, mine.budget, src);
        if (n_wide > 0) {
            __syncwarp();
            if (lane == 0) stk[0] = make_float2(0.0f, __int_as_float(0));
            __syncwarp();
            int top = 1;
            int budget = cap > 0 ? cap : n_wide;
            while (top > 0) {
                const float2 e = stk[top - 1];
                --top;
                if (!within(e.x, b2)) continue;                // pruned by a closer leaf found since
                if (--budget < 0) { err |= 1; break; }
                const float* f = wn + (size_t)__float_as_int(e.y) * WideLayout<DIM>::kFloats;
                float lo[DIM], hi[DIM], vt[DIM * DIM];
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    lo[k] = __ldg(f + k * kWide + lane);
                    hi[k] = __ldg(f + (DIM + k) * kWide + lane);
                }
                const int code = __float_as_int(__ldg(f + 2 * DIM * kWide + lane));
#pragma unroll
                for (int k = 0; k < DIM * DIM; ++k) vt[k] = __ldg(f + WideLayout<DIM>::kVtx + k * kWide + lane);
                const float cd = box_dist2<DIM>(q, lo, hi);
                if (lane == 0) ++n_nodes;
                const bool leaf = code < 0 && within(cd, b2);
                const unsigned lm = __ballot_sync(kWarpAll, leaf);
                if (lm) {
                    float dd = kInf;
                    if (leaf) {
                        if (DIM == 2) {
                            float t;
                            dd = seg_closest(q, vt[0], vt[1], vt[2], vt[3], t);
                        } else {
                            float w1, w2;
                            dd = tri_closest(q, make_float3(vt[0], vt[1], vt[2]), make_float3(vt[3], vt[4], vt[5]),
                                             make_float3(vt[6], vt[7], vt[8]), w1, w2);
                        }
                    }
                    // warp argmin, ties to the lower leaf index: squared distances are >= 0 (or
                    // +inf), so their bit patterns order like the values and one integer
                    // reduction finds the minimum; a second one picks the tied leaf
                    const unsigned bits = __float_as_uint(dd);
                    const unsigned mbits = __reduce_min_sync(kWarpAll, bits);
                    const unsigned pi = __reduce_min_sync(kWarpAll, leaf && bits == mbits ? (unsigned)~code : 0xffffffffu);
                    const float md = __uint_as_float(mbits);
                    if (closer(md, (int)pi, b2, bi)) { b2 = md; bi = (int)pi; }
                }
                const bool inner = code >= 0 && code != kEmptyChild && within(cd, b2);
                const unsigned im = __ballot_sync(kWarpAll, inner);
                if (im) {
                    const int cnt = __popc(im);
                    if (top + cnt > kWideStack) { err |= 4; break; }
                    // the nearest child (ties to the lower lane) goes on top (popped next); its
                    // siblings below it in lane order, which is the Morton order of the subtrees
                    const unsigned cbits = inner ? __float_as_uint(cd) : 0xffffffffu;
                    const unsigned mc = __reduce_min_sync(kWarpAll, cbits);
                    const int ml = __ffs(__ballot_sync(kWarpAll, inner && cbits == mc)) - 1;
                    const unsigned rest = im & ~(1u << ml);
                    __syncwarp();
                    if (inner) {
                        const int pos = lane == ml ? cnt - 1 : __popc(rest & ((1u << lane) - 1u));
                        stk[top + pos] = make_float2(cd, __int_as_float(code));
                    }
                    top += cnt;
                    __syncwarp();
                }
            }
        } else if (n_tree == 1) {
            const float dd = prim_dist2<DIM>(prims, 0, q);
            if (lane == 0) ++n_prims;
            if (closer(dd, 0, b2, bi)) { b2 = dd; bi = 0; }
        }
        if (lane == src) { best2 = b2; best = bi; }
    }
    return err;
}

// Outsized elements (kept out of the tree) against one lane's query.
template <int DIM>
__device__ __forceinline__ void big_closest(const float4* __restrict__ prims, int n_tree, int n_big, const float* q,
                                            float& best2, int& best, unsigned& n_prims) {
    for (int p = n_tree; p < n_tree + n_big; ++p) {
        if (!within(prim_box_dist2<DIM>(prims, p, q), best2)) continue;
        ++n_prims;
        const float dd = prim_dist2<DIM>(prims, p, q);
        if (closer(dd, p, best2, best)) { best2 = dd; best = p; }
    }
}

}  // namespace dwos
