// Persistent walk-on-spheres kernel (Algorithms 1 and 2 of "Differential Walk
// on Spheres", Miller et al. 2024).
//
// Each lane owns one walk at a time.  Every iteration of the loop is one
// distance query (DistanceToBoundary) for every busy lane of the warp,
// whatever phase its walk is in: the main walk (forward Algorithm 1, or the
// differential Algorithm 2 that also returns u from the same path), or one of
// its K nested forward walks from the offset point xbar - h n.  A lane whose
// walk ends writes its 32-byte record and takes the next walk from a global
// counter; the lanes of a warp that need work claim consecutive walk indices
// with one atomic (warp-aggregated refill), so a warp mostly works on walks
// of the same query point.  Walk state lives in registers; the problem
// descriptors live in shared memory.
//
// Randomness is Philox4x32-10 keyed by the seed, counter (walk id, step,
// phase << 8 | block): block 0 gives the sphere direction and the roulette
// draw, block 1 the ball sample of the source term.  Any walk can be replayed
// from its id alone.
#include "dwos_device.cuh"
#include "dwos_internal.h"
#include "wost.cuh"

namespace dwos {

namespace {

constexpr int kMaxProblems = 64;
constexpr unsigned kFull = 0xffffffffu;
// Search order 3 routes each query by the binary root's two child boxes: most
// queries (closer to an outsized element, or to their seed, than to any tree
// box) need no tree search at all; the few that do are searched by the whole
// warp over the 32-wide tree, one at a time, unless more than this many lanes
// of the warp need one in the same step, when each searches the binary tree.
constexpr int kRouteWideMax2 = 16;   // segments
constexpr int kRouteWideMax3 = 32;   // triangles: the per-lane binary search never pays

template <int DIM>
__device__ __forceinline__ float field_value(const float* c, const float* x, float* grad) {
    // g = c0 + c.x + x^T A x with A = [[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]]
    const float X = x[0], Y = x[1], Z = DIM == 3 ? x[2] : 0.0f;
    const float ax = c[4] * X + c[7] * Y + c[8] * Z;
    const float ay = c[7] * X + c[5] * Y + c[9] * Z;
    const float az = c[8] * X + c[9] * Y + c[6] * Z;
    grad[0] = c[1] + 2.0f * ax;
    grad[1] = c[2] + 2.0f * ay;
    if (DIM == 3) grad[2] = c[3] + 2.0f * az;
    return c[0] + c[1] * X + c[2] * Y + c[3] * Z + X * ax + Y * ay + Z * az;
}

// Closest point xbar on leaf `leaf`, its vertex weights, and the leaf's
// vertices (input order of the element).
template <int DIM>
__device__ __forceinline__ void leaf_geometry(const float4* __restrict__ prims, int leaf, const float* x,
                                              float* xbar, float& w1, float& w2, float* va, float* vb,
                                              float* vc) {
    if (DIM == 2) {
        const float4 s = __ldg(prims + leaf);
        va[0] = s.x; va[1] = s.y; vb[0] = s.z; vb[1] = s.w;
        seg_closest(x, s.x, s.y, s.z, s.w, w1);
        w2 = 0.0f;
        xbar[0] = fmaf(w1, s.z - s.x, s.x);
        xbar[1] = fmaf(w1, s.w - s.y, s.y);
    } else {
        const float4 a = __ldg(prims + 3 * leaf), b = __ldg(prims + 3 * leaf + 1), c = __ldg(prims + 3 * leaf + 2);
        va[0] = a.x; va[1] = a.y; va[2] = a.z;
        vb[0] = b.x; vb[1] = b.y; vb[2] = b.z;
        vc[0] = c.x; vc[1] = c.y; vc[2] = c.z;
        tri_closest(x, make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z), make_float3(c.x, c.y, c.z), w1, w2);
#pragma unroll
        for (int k = 0; k < 3; ++k) xbar[k] = va[k] + w1 * (vb[k] - va[k]) + w2 * (vc[k] - va[k]);
    }
}

struct WarpStats {             // per lane; summed over the warp in 64 bits at the end
    unsigned steps_main = 0, steps_nested = 0, capped = 0;
    unsigned nodes = 0, prims = 0, wnodes = 0;
};

// What a walk keeps from the end of its main walk until its last nested walk
// ends (read and written only at phase changes).  The warp-wide kernel keeps
// it in shared memory (an odd word count per thread: no bank conflicts) to
// leave the registers to the search; the per-lane kernels keep it in registers.
template <int DIM>
struct PhaseState {
    float u_main, g_main, b1, b2;
    float sum_plain, sum_dn, sum_dt;     // nested walks: estimates, n / t displacements
    float sum_ball, w_ball;              // ball-gradient estimator: weighted sum, this nested walk's weight
    float nrm[DIM], cb[DIM], xoff[DIM];
    int leaf_main, e_main;
    uint32_t meta_main;
    uint32_t pad[DIM == 2 ? 1 : 2];      // 19 / 23 words
};

// Dynamic shared memory: the problem descriptors, then (warp-wide search only)
// one traversal stack per warp and the threads' phase states, or (walk on
// stars) the Neumann part's descriptor.
__host__ __device__ inline size_t walk_smem_bytes(int n_probs, int block_size, int traversal, int dim = 3,
                                                  bool star = false) {
    size_t b = (sizeof(DevProblem) * (size_t)n_probs + 15) & ~(size_t)15;
    if (traversal == 2 || traversal == 3)
        b += sizeof(float2) * kWideStack * (size_t)(block_size / 32) +
             (dim == 2 ? sizeof(PhaseState<2>) : sizeof(PhaseState<3>)) * (size_t)block_size;
    if (star) b += sizeof(DevNeumann);
    return b;
}

// Uniform direction on the unit circle / sphere from words 0 (and 1) of a block.
template <int DIM>
__device__ __forceinline__ void sphere_dir(const U4& r, float* om) {
    if (DIM == 2) {
        float s, c;
        sincospif(2.0f * u01(r.x), &s, &c);
        om[0] = c; om[1] = s; om[2] = 0.0f;
    } else {
        const float u0 = u01(r.x);
        const float z = 1.0f - 2.0f * u0;
        const float sth = 2.0f * sqrtf(u0 * (1.0f - u0));
        float s, c;
        sincospif(2.0f * u01(r.y), &s, &c);
        om[0] = sth * c; om[1] = sth * s; om[2] = z;
    }
}

// STAR: walk on stars over a boundary with a Neumann part (one problem per
// launch; the Dirichlet part's distance queries take the launch's search
// order, the Neumann queries per lane).  DATA: the Neumann part carries data
// du/dn (a separate instantiation, so that reflecting walks keep their code).
template <int DIM, bool WIDE, bool STAR = false, bool CONES = false, bool DATA = false>
__global__ void __launch_bounds__(256, STAR ? 3 : ((DIM == 2 || WIDE) ? 4 : 3))
    walk_kernel(const DevProblem* __restrict__ g_probs, int n_probs, unsigned long long total,
                DevCounters* __restrict__ ctr, DevCounters* __restrict__ zero_ctr,
                const __grid_constant__ DevProblem p_arg) {
    constexpr bool wide = WIDE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DevProblem* sp = reinterpret_cast<DevProblem*>(smem_raw);
    float2* stk_base = reinterpret_cast<float2*>(smem_raw + walk_smem_bytes(n_probs, 0, 0));
    float2* stk = stk_base + (size_t)(threadIdx.x >> 5) * kWideStack;
    PhaseState<DIM> ps_reg;
    PhaseState<DIM>& S = WIDE ? reinterpret_cast<PhaseState<DIM>*>(stk_base + (size_t)(blockDim.x >> 5) * kWideStack)[threadIdx.x]
                              : ps_reg;
    {
        // the descriptor table, or the one problem passed by value
        const int words = (int)(sizeof(DevProblem) / sizeof(int)) * n_probs;
        const int* src = g_probs ? reinterpret_cast<const int*>(g_probs) : reinterpret_cast<const int*>(&p_arg);
        int* dst = reinterpret_cast<int*>(sp);
        for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
        // the counters of the next launch start at zero
        if (zero_ctr && blockIdx.x == 0)
            for (int i = threadIdx.x; i < (int)(sizeof(DevCounters) / sizeof(int)); i += blockDim.x)
                reinterpret_cast<int*>(zero_ctr)[i] = 0;
    }
    __syncthreads();
    // the Neumann descriptor follows the problems (and, warp-wide, the stacks and phase states)
    DevNeumann& NS = *reinterpret_cast<DevNeumann*>(smem_raw + walk_smem_bytes(n_probs, WIDE ? (int)blockDim.x : 0,
                                                                               WIDE ? 3 : 0, DIM, false));
    if constexpr (STAR) {
        const int words = (int)(sizeof(DevNeumann) / sizeof(int));
        const int* src = reinterpret_cast<const int*>(sp[0].neu);
        int* dst = reinterpret_cast<int*>(&NS);
        for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
        __syncthreads();
    }
    int on_e = -1;                  // STAR: the Neumann element the walk sits on (compact), -1 inside
    float n_on[DIM];                // STAR: its normal, out of the domain
    int on2 = -1;                   // STAR: at an edge, the side it came from and still lies on
    float n2[DIM];                  // STAR: that side's normal, out of the domain
    int nst1 = -1, nst2 = -1;       // STAR: the sides the nested walks start on, 2 e + (normal flipped)
#pragma unroll
    for (int k = 0; k < DIM; ++k) { n_on[k] = 0.0f; n2[k] = 0.0f; }

    const int lane = threadIdx.x & 31;
    bool active = false, exhausted = false;
    int error = 0;
    WarpStats st;

    // per-lane walk state
    unsigned long long gw = 0;      // global work index of the current walk
    int prob = 0, phase = 0, step = 0, hint = -1;
    float x[DIM], acc = 0.0f;
    // main-walk results kept while the nested walks run
    S.u_main = 0.0f; S.g_main = 0.0f; S.b1 = 0.0f; S.b2 = 0.0f;
    S.sum_plain = 0.0f; S.sum_dn = 0.0f; S.sum_dt = 0.0f; S.sum_ball = 0.0f; S.w_ball = 0.0f;
    S.leaf_main = -1; S.e_main = -1; S.meta_main = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) { x[k] = 0.0f; S.nrm[k] = 0.0f; S.cb[k] = 0.0f; S.xoff[k] = 0.0f; }

    for (;;) {
        // ---- refill idle lanes with consecutive walk indices (one atomic per warp)
        const unsigned need = __ballot_sync(kFull, !active && !exhausted);
        if (need) {
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(&ctr->next_work, (unsigned long long)__popc(need));
            base = __shfl_sync(kFull, base, leader);
            if (!active && !exhausted) {
                const unsigned long long my = base + __popc(need & ((1u << lane) - 1u));
                if (my < total) {
                    gw = my;
                    while (prob + 1 < n_probs && gw >= sp[prob].work_end) ++prob;
                    const DevProblem& P = sp[prob];
                    const unsigned long long local = gw - P.work_begin;
                    const int point = (int)(local / (unsigned long long)P.walks);
                    bool finite = true;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) {
                        x[k] = __ldg(P.xq + (size_t)DIM * point + k);
                        finite = finite && isfinite(x[k]);
                    }
                    if (!finite || (P.valid && !__ldg(P.valid + point))) {
                        // query point not finite (error bit 4) or outside Omega (bit 2): NaN record, next walk
                        dwos_record r;
                        r.u = __int_as_float(0x7fc00000); r.elem = -1; r.b1 = 0.0f; r.b2 = 0.0f;
                        r.c[0] = 0.0f; r.c[1] = 0.0f; r.c[2] = 0.0f; r.meta = 0;
                        P.rec[local] = r;
                        error |= finite ? 2 : 4;
                    } else {
                        phase = 0; step = 0; hint = -1; acc = 0.0f;
                        on_e = -1;
                        on2 = -1;
                        if constexpr (STAR) {   // a query point on the Neumann part starts on it
                            if (NS.q_start) {
                                const float4 qs = NS.q_start[point];
                                on_e = __float_as_int(qs.w);
                                n_on[0] = qs.x; n_on[1] = qs.y;
                                if (DIM == 3) n_on[DIM - 1] = qs.z;
                            }
                        }
                        active = true;
                    }
                } else {
                    exhausted = true;
                }
            }
        }
        if (!__any_sync(kFull, active)) break;

        // ---- DistanceToBoundary, seeded with the previous closest element
        float best2 = kInf;
        int best = -1;
        bool lane_search = !wide;
        bool seeded = false;   // hint and outsized elements already tested
        if (wide) {
            const DevProblem& Pw = sp[prob];
            if (active) {
                if (hint >= 0) { best2 = prim_dist2<DIM>(Pw.prims, hint, x); best = hint; ++st.prims; }
                big_closest<DIM>(Pw.prims, Pw.n_tree, Pw.n_big, x, best2, best, st.prims);
                seeded = true;
            }
            unsigned need = __ballot_sync(kFull, active);
            if (sp[0].traversal == 3) {   // the same order for every problem of a launch
                // route: only queries with a root child box inside the bound need the tree
                bool desc = false;
                if (active) {
                    if (Pw.n_internal > 0) {
                        float lo0[DIM], hi0[DIM], lo1[DIM], hi1[DIM];
                        int c0, c1, parent;
                        load_node<DIM>(Pw.nodes, Pw.root, lo0, hi0, lo1, hi1, c0, c1, parent);
                        ++st.nodes;
                        desc = within(box_dist2<DIM>(x, lo0, hi0), best2) || within(box_dist2<DIM>(x, lo1, hi1), best2);
                    } else {
                        desc = Pw.n_tree > 0;
                    }
                }
                need = __ballot_sync(kFull, desc);
                if (__popc(need) > (DIM == 2 ? kRouteWideMax2 : kRouteWideMax3)) {   // many searches this step: one per lane, in parallel
                    lane_search = desc;
                    need = 0;
                }
            }
            if (need) {   // all lanes search the 32-wide tree together, one lane's query at a time
                const WideView wv{Pw.wnodes, Pw.prims, Pw.n_wide, Pw.n_tree, Pw.node_budget};
                error |= wide_closest<DIM>(wv, need, x, best2, best, stk, st.wnodes, st.prims) & 1;
            }
        }
        if (!active) continue;

        const DevProblem& P = sp[prob];
        const unsigned long long local = gw - P.work_begin;
        if (lane_search) {
            BvhView bvh{P.nodes, P.prims, P.root, P.n_internal, P.n_tree, seeded ? 0 : P.n_big, P.traversal == 1,
                        P.leaf_parent, P.node_cell, P.r_max, P.node_budget};
            if (!seeded && hint >= 0) { best2 = prim_dist2<DIM>(P.prims, hint, x); best = hint; ++st.prims; }
            if (!closest_leaf<DIM>(bvh, x, best2, best, st.nodes, st.prims)) error |= 1;
        }
        const float d = sqrtf(best2);
        const uint32_t k_step = (uint32_t)step;
        ++step;
        if (phase == 0) ++st.steps_main; else ++st.steps_nested;

        bool lost = best < 0;   // only with non-finite geometry or points: end the walk
        if constexpr (STAR) lost = lost || !(best2 < kInf);   // a walk that left the domain
        const bool shell = !lost && d < P.eps;
        const bool capped = !lost && !shell && step >= P.max_steps;
        int kind;
        float g = 0.0f;
        float xbar[DIM], w1 = 0.0f, w2 = 0.0f, va[DIM], vb[DIM], vc[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) { xbar[k] = 0.0f; va[k] = 0.0f; vb[k] = 0.0f; vc[k] = 0.0f; }
        int e = -1;
        if (lost) {
            error |= 1;
            kind = DWOS_KIND_ROULETTE;
        } else if (shell || capped) {
            kind = shell ? DWOS_KIND_SHELL : DWOS_KIND_CAPPED;
            if (capped) ++st.capped;
            leaf_geometry<DIM>(P.prims, best, x, xbar, w1, w2, va, vb, vc);
            e = __ldg(P.prim_elem + best);
            if constexpr (STAR) e = __ldg(NS.dmap + e);      // the Dirichlet BVH numbers its own elements
            if (P.data_kind == 1) {
                float gr[DIM];
                g = field_value<DIM>(P.field, xbar, gr);
            } else {
                const int* ev = P.elem + (size_t)DIM * e;
                const float w0 = 1.0f - w1 - w2;
                g = w0 * __ldg(P.g_vert + ev[0]) + w1 * __ldg(P.g_vert + ev[1]);
                if (DIM == 3) g += w2 * __ldg(P.g_vert + ev[2]);
            }
        } else if constexpr (STAR) {
            // walk on stars: R from the Dirichlet distance and the Neumann silhouettes
            const unsigned long long wid = P.walk_id_base + local;
            bool ok1 = true, ok2 = true, ok3 = true;
            const float sd2 = silhouette_dist2<DIM, CONES>(NS, x, best2, on_e, on2, ok1);
            // R = max(min(d_D - c, d_sil), eps - c), c = 1e-3 eps the Dirichlet clearance
            const float R = fmaxf(fminf(sqrtf(sd2), fmaf(-1e-3f, P.eps, d)), fmaf(-1e-3f, P.eps, P.eps));
            if (P.f != 0.0f) {   // source: a point of the ball, counted if x sees it
                const U4 r1 = draw_block(P.seed_lo, P.seed_hi, wid, k_step, (uint32_t)phase, 1u);
                float w[3];
                sphere_dir<DIM>(r1, w);
                turn_inward<DIM>(w, on_e, n_on, on2, n2);
                const float ub = u01(r1.z);
                const float rr = R * (DIM == 2 ? sqrtf(ub) : cbrtf(ub));
                int h2;
                ray_neumann<DIM>(NS, x, w, rr, on_e, n_on, on2, n2, 1e-4f * P.eps, h2, ok2);
                if (h2 < 0) acc = fmaf(source_weight<DIM>(P.sqrt_sigma, R, ub), P.f, acc);
            }
            if constexpr (DATA) {   // Neumann data: a point of the Neumann part in the ball, counted if x sees it
                Vec3 xv{{0.0f, 0.0f, 0.0f}}, nv{{0.0f, 0.0f, 0.0f}}, mv{{0.0f, 0.0f, 0.0f}};
#pragma unroll
                for (int i = 0; i < DIM; ++i) { xv.v[i] = x[i]; nv.v[i] = n_on[i]; mv.v[i] = n2[i]; }
                const DataSample ds = neumann_data_sample<DIM>(NS, xv, R, on_e, nv, on2, mv, 1e-4f * P.eps,
                                                               P.sqrt_sigma, P.seed_lo, P.seed_hi, wid, k_step,
                                                               (uint32_t)phase);
                acc += ds.w;
                if (!ds.ok) ok2 = false;
            }
            const U4 r0 = draw_block(P.seed_lo, P.seed_hi, wid, k_step, (uint32_t)phase, 0u);
            float om[3];
            sphere_dir<DIM>(r0, om);
            turn_inward<DIM>(om, on_e, n_on, on2, n2);   // on the Neumann part: into the domain
            int hit;
            const float th = ray_neumann<DIM>(NS, x, om, R, on_e, n_on, on2, n2, 1e-4f * P.eps, hit, ok3);
            if (!(ok1 && ok2 && ok3)) error |= 1;
            const float t = hit >= 0 ? th : R;
            if (P.sqrt_sigma > 0.0f && star_weight<DIM>(P.sqrt_sigma, t, R) < u01(r0.z)) {
                kind = DWOS_KIND_ROULETTE;
            } else {
#pragma unroll
                for (int k = 0; k < DIM; ++k) x[k] = fmaf(t, om[k], x[k]);
                // a move that leaves a side by at most 1e-4 eps along its normal (a direction
                // nearly tangent to it) leaves the walk on that side
                float s1 = 0.0f, s2 = 0.0f;
#pragma unroll
                for (int k = 0; k < DIM; ++k) { s1 = fmaf(om[k], n_on[k], s1); s2 = fmaf(om[k], n2[k], s2); }
                const bool keep = on_e >= 0 && fabsf(t * s1) <= 1e-4f * P.eps;
                const bool keep2 = on2 >= 0 && fabsf(t * s2) <= 1e-4f * P.eps;
                if (hit >= 0) {
                    // on the element hit, and on an edge if still on the side it left; the hit
                    // element's normal, oriented along the ray (out of the domain)
                    on2 = keep ? on_e : -1;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) n2[k] = n_on[k];
                    neumann_normal<DIM>(NS, hit, n_on);
                    float s = 0.0f;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) s = fmaf(n_on[k], om[k], s);
                    if (s < 0.0f) {
#pragma unroll
                        for (int k = 0; k < DIM; ++k) n_on[k] = -n_on[k];
                    }
                    on_e = hit;
                } else if (keep) {
                    if (!keep2) on2 = -1;
                } else if (keep2) {
                    on_e = on2;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) n_on[k] = n2[k];
                    on2 = -1;
                } else {
                    on_e = -1;
                    on2 = -1;
                }
                hint = best;
                continue;
            }
        } else {
            const unsigned long long wid = P.walk_id_base + local;
            // ball-gradient estimator: a nested walk's first move samples y on the sphere
            // about the offset point (no source, no roulette) and weighs the estimate at y
            const bool ball = P.dudn_mode == 1 && phase > 0 && k_step == 0;
            // the ball keeps a clearance of 1e-3 eps from the boundary: the landing point stays on
            // the domain's side by more than FP32 rounding (any ball inside the domain is a valid step)
            const float rs = fmaf(-1e-3f, P.eps, d);
            if (P.f != 0.0f && !ball) {   // source estimate of this ball (Algorithm 1, S-hat)
                const U4 r1 = draw_block(P.seed_lo, P.seed_hi, wid, k_step, (uint32_t)phase, 1u);
                acc = fmaf(source_weight<DIM>(P.sqrt_sigma, rs, u01(r1.z)), P.f, acc);
            }
            const U4 r0 = draw_block(P.seed_lo, P.seed_hi, wid, k_step, (uint32_t)phase, 0u);
            if (!ball && roulette_stops<DIM>(P.sqrt_sigma, rs, u01(r0.z))) {
                kind = DWOS_KIND_ROULETTE;
            } else {   // next point on the sphere of radius rs
                float om[3];
                if (DIM == 2) {
                    float s, c;
                    sincospif(2.0f * u01(r0.x), &s, &c);
                    om[0] = c; om[1] = s; om[2] = 0.0f;
                } else {
                    const float u0 = u01(r0.x);
                    const float z = 1.0f - 2.0f * u0;
                    const float sth = 2.0f * sqrtf(u0 * (1.0f - u0));
                    float s, c;
                    sincospif(2.0f * u01(r0.y), &s, &c);
                    om[0] = sth * c; om[1] = sth * s; om[2] = z;
                }
#pragma unroll
                for (int k = 0; k < DIM; ++k) x[k] = fmaf(rs, om[k], x[k]);
                if (ball) {
                    float on = 0.0f;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) on = fmaf(om[k], S.nrm[k], on);
                    S.w_ball = gradient_factor<DIM>(P.sqrt_sigma, rs) * on;
                }
                hint = best;
                if (phase == 0 && k_step == 0 && P.cv_sample)   // first step of the main walk
                    P.cv_sample[local] = make_float4(x[0], x[1], DIM == 3 ? x[DIM - 1] : 0.0f, acc);
                continue;
            }
        }

        // ---- the current phase ended (shell, capped or roulette)
        const int K1 = P.K + 1;
        if (P.trace) P.trace[local * K1 + phase] = min((uint32_t)step, 0x3fffffffu) | ((uint32_t)kind << 30);
        if (phase == 0) {
            if (P.cv_end) P.cv_end[local] = make_float4(x[0], x[1], DIM == 3 ? x[DIM - 1] : 0.0f, 0.0f);
            S.u_main = acc + g;
            S.meta_main = min((uint32_t)step, 0xffffffu) | ((uint32_t)kind << 24);
            if (!P.differential || kind == DWOS_KIND_ROULETTE) {
                dwos_record r;
                r.u = S.u_main;
                r.elem = kind == DWOS_KIND_ROULETTE ? -1 : e;
                r.b1 = w1; r.b2 = w2;
                r.c[0] = 0.0f; r.c[1] = 0.0f; r.c[2] = 0.0f;
                r.meta = S.meta_main;
                P.rec[local] = r;
                if (P.differential) {
                    if (P.trace) for (int j = 1; j < K1; ++j) P.trace[local * K1 + j] = 0xffffffffu;
                    if (P.dbg) {
                        dwos_walk_debug z;
                        z.dudn = 0.0f; z.u_off = 0.0f;
                        for (int k = 0; k < 3; ++k) { z.n[k] = 0.0f; z.xbar[k] = k < DIM ? xbar[k] * (kind != DWOS_KIND_ROULETTE) : 0.0f; }
                        z.u_plain = 0.0f; z.disp_n = 0.0f; z.disp_t = 0.0f;
                        z.elem = kind == DWOS_KIND_ROULETTE ? -1 : e;
                        P.dbg[local] = z;
                    }
                }
                active = false;
                continue;
            }
            // BoundaryNormal at xbar, oriented away from the walk point (Algorithm 2)
            float side = 0.0f;
            if (DIM == 2) {
                const float tx = vb[0] - va[0], ty = vb[1] - va[1];
                const float inv = rsqrtf(tx * tx + ty * ty);
                S.nrm[0] = ty * inv;
                S.nrm[1] = -tx * inv;
            } else {
                const float e1[3] = {vb[0] - va[0], vb[1] - va[1], vb[2] - va[2]};
                const float e2[3] = {vc[0] - va[0], vc[1] - va[1], vc[2] - va[2]};
                const float cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                     e1[0] * e2[1] - e1[1] * e2[0]};
                const float inv = rsqrtf(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
                S.nrm[0] = cr[0] * inv; S.nrm[1] = cr[1] * inv; S.nrm[DIM - 1] = cr[2] * inv;
            }
#pragma unroll
            for (int k = 0; k < DIM; ++k) side = fmaf(S.nrm[k], xbar[k] - x[k], side);
            if (side < 0.0f) {
#pragma unroll
                for (int k = 0; k < DIM; ++k) S.nrm[k] = -S.nrm[k];
            }
            // boundary-data part of c: (dg/dn) n for field data (Eq. boundary_deriv_restricted),
            // -grad_Gamma(g) for mapped data (Eq. boundary_deriv_mapped with dg/dn = 0)
            if (P.data_kind == 1) {
                float gr[DIM];
                field_value<DIM>(P.field, xbar, gr);
                float dgdn = 0.0f;
#pragma unroll
                for (int k = 0; k < DIM; ++k) dgdn = fmaf(S.nrm[k], gr[k], dgdn);
#pragma unroll
                for (int k = 0; k < DIM; ++k) S.cb[k] = dgdn * S.nrm[k];
            } else {
                const int* ev = P.elem + (size_t)DIM * e;
                const float g0 = __ldg(P.g_vert + ev[0]);
                if (DIM == 2) {
                    const float tx = vb[0] - va[0], ty = vb[1] - va[1];
                    const float s = (__ldg(P.g_vert + ev[1]) - g0) / (tx * tx + ty * ty);
                    S.cb[0] = -s * tx;
                    S.cb[1] = -s * ty;
                } else {
                    const float e1[3] = {vb[0] - va[0], vb[1] - va[1], vb[2] - va[2]};
                    const float e2[3] = {vc[0] - va[0], vc[1] - va[1], vc[2] - va[2]};
                    const float g11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
                    const float g12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
                    const float g22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
                    const float r1 = __ldg(P.g_vert + ev[1]) - g0, r2 = __ldg(P.g_vert + ev[2]) - g0;
                    const float det = g11 * g22 - g12 * g12;
                    const float a1 = (g22 * r1 - g12 * r2) / det, a2 = (g11 * r2 - g12 * r1) / det;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) S.cb[k] = -(a1 * e1[k] + a2 * e2[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < DIM; ++k) S.xoff[k] = fmaf(-P.h, S.nrm[k], xbar[k]);
            if constexpr (STAR) {   // mirrored across the Neumann part where the offset crosses it
                float back[3] = {-S.nrm[0], -S.nrm[1], DIM == 3 ? -S.nrm[DIM - 1] : 0.0f};
                int he;
                bool okr = true;
                const float th = ray_neumann<DIM>(NS, xbar, back, P.h, -1, back, -1, back, 0.0f, he, okr);
                if (!okr) error |= 1;
                if (he >= 0) {
                    float m[3];
                    neumann_normal<DIM>(NS, he, m);
                    float c[DIM], r[DIM], rm = 0.0f;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) {
                        c[k] = fmaf(th, back[k], xbar[k]);
                        r[k] = S.xoff[k] - c[k];
                        rm = fmaf(r[k], m[k], rm);
                    }
#pragma unroll
                    for (int k = 0; k < DIM; ++k) S.xoff[k] = c[k] + fmaf(-2.0f * rm, m[k], r[k]);
                }
                // the nested walks start on the Neumann side(s) the main walk ended on where the
                // offset point lies on it (within 1e-4 eps of its plane)
                float r1 = 0.0f, r2 = 0.0f;
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    r1 = fmaf(S.xoff[k] - x[k], n_on[k], r1);
                    r2 = fmaf(S.xoff[k] - x[k], n2[k], r2);
                }
                const bool k1 = on_e >= 0 && fabsf(r1) <= 1e-4f * P.eps;
                const bool k2 = on2 >= 0 && fabsf(r2) <= 1e-4f * P.eps;
                auto code = [&](int e2, const float* n) {
                    float m[3] = {0.0f, 0.0f, 0.0f}, sg = 0.0f;
                    neumann_normal<DIM>(NS, e2, m);
#pragma unroll
                    for (int k = 0; k < DIM; ++k) sg = fmaf(m[k], n[k], sg);
                    return 2 * e2 + (sg < 0.0f ? 1 : 0);
                };
                nst1 = k1 ? code(on_e, n_on) : (k2 ? code(on2, n2) : -1);
                nst2 = k1 && k2 ? code(on2, n2) : -1;
            }
            S.g_main = g; S.b1 = w1; S.b2 = w2; S.leaf_main = best; S.e_main = e;
            S.sum_plain = 0.0f; S.sum_dn = 0.0f; S.sum_dt = 0.0f; S.sum_ball = 0.0f; S.w_ball = 0.0f;
        } else {
            // nested control variate: (q n + t) . (x_end - x_off) has mean zero (every
            // move's direction is uniform and independent of whether the move happens)
            float dn = 0.0f, dt = 0.0f;
#pragma unroll
            for (int k = 0; k < DIM; ++k) dn = fmaf(S.nrm[k], x[k] - S.xoff[k], dn);
            float q = 0.0f;
            if (P.cv_elem) {
                const float4 qc = __ldg(P.cv_elem + S.e_main);
                const float tv[3] = {qc.y, qc.z, qc.w};
#pragma unroll
                for (int k = 0; k < DIM; ++k) dt = fmaf(tv[k], x[k] - S.xoff[k], dt);
                q = qc.x;
            }
            S.sum_plain += acc + g;
            S.sum_dn += dn;
            S.sum_dt += dt;
            S.sum_ball = fmaf(S.w_ball, acc + g, S.sum_ball);   // zero unless the ball estimator moved
            S.w_ball = 0.0f;
            if (phase == P.K) {   // Eq. (wos_deriv), shell case, with Eq. (dudn_fd_estimate) or (dudn_mc_estimate)
                const float inv_k = 1.0f / (float)P.K;
                const float u_off = (S.sum_plain - fmaf(q, S.sum_dn, S.sum_dt)) * inv_k;
                const float dudn = P.dudn_mode == 1 ? S.sum_ball * inv_k : (S.g_main - u_off) * P.inv_h;
                dwos_record r;
                r.u = S.u_main;
                r.elem = S.e_main;
                r.b1 = S.b1; r.b2 = S.b2;
                r.c[0] = S.cb[0] - dudn * S.nrm[0];
                r.c[1] = S.cb[1] - dudn * S.nrm[1];
                r.c[2] = DIM == 3 ? S.cb[DIM - 1] - dudn * S.nrm[DIM - 1] : 0.0f;
                r.meta = S.meta_main;
                P.rec[local] = r;
                if (P.dbg) {
                    dwos_walk_debug z;
                    z.dudn = dudn;
                    z.u_off = u_off;
                    for (int k = 0; k < 3; ++k) {
                        z.n[k] = k < DIM ? S.nrm[k] : 0.0f;
                        z.xbar[k] = k < DIM ? fmaf(P.h, S.nrm[k], S.xoff[k]) : 0.0f;
                    }
                    z.u_plain = S.sum_plain * inv_k;
                    z.disp_n = S.sum_dn * inv_k;
                    z.disp_t = S.sum_dt * inv_k;
                    z.elem = S.e_main;
                    P.dbg[local] = z;
                }
                active = false;
                continue;
            }
        }
        // start the next nested forward walk from the offset point
        ++phase;
        step = 0;
        acc = 0.0f;
        on_e = -1;
        on2 = -1;
        if constexpr (STAR) {   // on the side(s) the main walk ended on, where the offset point lies on them
            if (nst1 >= 0) {
                on_e = nst1 >> 1;
                neumann_normal<DIM>(NS, on_e, n_on);
                if (nst1 & 1) {
#pragma unroll
                    for (int k = 0; k < DIM; ++k) n_on[k] = -n_on[k];
                }
            }
            if (nst2 >= 0) {
                on2 = nst2 >> 1;
                neumann_normal<DIM>(NS, on2, n2);
                if (nst2 & 1) {
#pragma unroll
                    for (int k = 0; k < DIM; ++k) n2[k] = -n2[k];
                }
            }
        }
        hint = S.leaf_main;
#pragma unroll
        for (int k = 0; k < DIM; ++k) x[k] = S.xoff[k];
    }

    // ---- statistics: one atomic per warp
    unsigned long long sm = st.steps_main, sn = st.steps_nested, sc = st.capped;
    for (int o = 16; o > 0; o >>= 1) {
        sm += __shfl_xor_sync(kFull, sm, o);
        sn += __shfl_xor_sync(kFull, sn, o);
        sc += __shfl_xor_sync(kFull, sc, o);
        error |= __shfl_xor_sync(kFull, error, o);
    }
    unsigned long long nodes = st.nodes, prims = st.prims, wnodes = st.wnodes;
    for (int o = 16; o > 0; o >>= 1) {
        nodes += __shfl_xor_sync(kFull, nodes, o);
        prims += __shfl_xor_sync(kFull, prims, o);
        wnodes += __shfl_xor_sync(kFull, wnodes, o);
    }
    if (lane == 0) {
        atomicAdd(&ctr->steps_main, sm);
        atomicAdd(&ctr->steps_nested, sn);
        atomicAdd(&ctr->nodes, nodes);
        atomicAdd(&ctr->prims, prims);
        if (wnodes) atomicAdd(&ctr->wnodes, wnodes);
        if (sc) atomicAdd(&ctr->capped, sc);
        if (error) atomicOr(&ctr->error, error);
    }
}

// The ball weights of one walk step, exactly as the walk kernel evaluates them:
// the source factor |B(d)| G_d(r) for the ball sample drawn from the uniform u,
// and the recursive weight alpha(d).
template <int DIM>
__global__ void ball_weights_kernel(float k, int n, const float* __restrict__ d, const float* __restrict__ u,
                                    float* __restrict__ src, float* __restrict__ alpha) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (src) src[i] = source_weight<DIM>(k, d[i], u[i]);
    if (alpha) alpha[i] = recursive_weight<DIM>(k, d[i]);
}

__global__ void bessel_k_kernel(int order, int n, const float* __restrict__ x, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = order == 0 ? bessel_k0(x[i]) : bessel_k1(x[i]);
}

template <int DIM>
__global__ void star_weight_kernel(float k, int n, const float* __restrict__ t, const float* __restrict__ R,
                                   float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = star_weight<DIM>(k, t[i], R[i]);
}

}  // namespace

cudaError_t launch_ball_weights(int dim, float k, int n, const float* d, const float* u, float* src, float* alpha,
                                cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (n + 255) / 256;
    if (dim == 2) ball_weights_kernel<2><<<blocks, 256, 0, stream>>>(k, n, d, u, src, alpha);
    else ball_weights_kernel<3><<<blocks, 256, 0, stream>>>(k, n, d, u, src, alpha);
    return cudaGetLastError();
}

cudaError_t launch_bessel_k(int order, int n, const float* x, float* out, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    bessel_k_kernel<<<(n + 255) / 256, 256, 0, stream>>>(order, n, x, out);
    return cudaGetLastError();
}

cudaError_t launch_star_weight(int dim, float k, int n, const float* t, const float* R, float* out, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    if (dim == 2) star_weight_kernel<2><<<(n + 255) / 256, 256, 0, stream>>>(k, n, t, R, out);
    else star_weight_kernel<3><<<(n + 255) / 256, 256, 0, stream>>>(k, n, t, R, out);
    return cudaGetLastError();
}

namespace {

template <int DIM>
__global__ void neumann_start_kernel(int n, const float* __restrict__ xq, DevNeumann N, float tol2,
                                     float4* __restrict__ q_start, float* __restrict__ behind) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float x[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) x[k] = xq[DIM * p + k];
    BvhView bvh{N.nodes, N.prims, 0, N.n_internal, N.n_tree, N.n_big, 0, nullptr, nullptr, 0.0f};
    float best2 = kInf;
    int best = -1;
    unsigned nn = 0, np = 0;
    closest_leaf<DIM>(bvh, x, best2, best, nn, np);
    float4 out = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(-1));
#pragma unroll
    for (int k = 0; k < DIM; ++k) behind[DIM * p + k] = x[k];
    if (best >= 0 && best2 <= tol2) {
        const int e = __ldg(N.prim_elem + best);
        float m[3] = {0.0f, 0.0f, 0.0f};
        neumann_normal<DIM>(N, e, m);
        float a[DIM], b[DIM], c[DIM], size;
        const int* ev = N.elem + (size_t)DIM * e;
        vload<DIM>(N.vert, __ldg(ev), a);
        vload<DIM>(N.vert, __ldg(ev + 1), b);
        if (DIM == 2) {
            size = sqrtf((b[0] - a[0]) * (b[0] - a[0]) + (b[1] - a[1]) * (b[1] - a[1]));
#pragma unroll
            for (int k = 0; k < DIM; ++k) c[k] = 0.5f * (a[k] + b[k]);
        } else {
            float v[DIM];
            vload<DIM>(N.vert, __ldg(ev + 2), v);
            const float u1[3] = {b[0] - a[0], b[1] - a[1], b[DIM - 1] - a[DIM - 1]};
            const float u2[3] = {v[0] - a[0], v[1] - a[1], v[DIM - 1] - a[DIM - 1]};
            const float w0 = u1[1] * u2[2] - u1[2] * u2[1], w1 = u1[2] * u2[0] - u1[0] * u2[2],
                        w2 = u1[0] * u2[1] - u1[1] * u2[0];
            size = sqrtf(sqrtf(w0 * w0 + w1 * w1 + w2 * w2));
#pragma unroll
            for (int k = 0; k < DIM; ++k) c[k] = (a[k] + b[k] + v[k]) * (1.0f / 3.0f);
        }
#pragma unroll
        for (int k = 0; k < DIM; ++k) behind[DIM * p + k] = c[k] - 1e-3f * size * m[k];
        out = make_float4(m[0], m[1], m[2], __int_as_float(e));
    }
    q_start[p] = out;
}

__global__ void neumann_orient_kernel(int n, const int* __restrict__ behind_inside, float4* __restrict__ q_start,
                                      int* __restrict__ valid) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float4 q = q_start[p];
    if (__float_as_int(q.w) < 0) return;
    if (!behind_inside[p]) { q.x = -q.x; q.y = -q.y; q.z = -q.z; }
    q_start[p] = q;
    if (valid) valid[p] = 1;     // on the boundary: ray parity says nothing there
}

}  // namespace

cudaError_t launch_neumann_start(int dim, int n, const float* xq, const DevNeumann& N, float tol,
                                 float4* q_start, float* behind, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (n + 127) / 128;
    if (dim == 2) neumann_start_kernel<2><<<blocks, 128, 0, s>>>(n, xq, N, tol * tol, q_start, behind);
    else neumann_start_kernel<3><<<blocks, 128, 0, s>>>(n, xq, N, tol * tol, q_start, behind);
    return cudaGetLastError();
}

cudaError_t launch_neumann_orient(int n, const int* behind_inside, float4* q_start, int* valid, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    neumann_orient_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, behind_inside, q_start, valid);
    return cudaGetLastError();
}

int walk_max_blocks_per_sm(int dim, int block_size, int traversal, bool star, bool cones, bool data) {
    int n = 0;
    const size_t smem = walk_smem_bytes(1, block_size, traversal, dim, star);
    const bool wide = traversal == 2 || traversal == 3;
    auto occ = [&](auto kernel) { cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block_size, smem); };
    if (star && data) {
        if (dim == 2) wide ? occ(walk_kernel<2, true, true, false, true>) : occ(walk_kernel<2, false, true, false, true>);
        else wide ? occ(walk_kernel<3, true, true, false, true>) : occ(walk_kernel<3, false, true, false, true>);
    } else if (star) {
        if (dim == 2) {
            if (wide) cones ? occ(walk_kernel<2, true, true, true>) : occ(walk_kernel<2, true, true>);
            else cones ? occ(walk_kernel<2, false, true, true>) : occ(walk_kernel<2, false, true>);
        } else {
            if (wide) cones ? occ(walk_kernel<3, true, true, true>) : occ(walk_kernel<3, true, true>);
            else cones ? occ(walk_kernel<3, false, true, true>) : occ(walk_kernel<3, false, true>);
        }
    } else if (traversal == 2 || traversal == 3) {
        if (dim == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, walk_kernel<2, true>, block_size, smem);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, walk_kernel<3, true>, block_size, smem);
    } else {
        if (dim == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, walk_kernel<2, false>, block_size, smem);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, walk_kernel<3, false>, block_size, smem);
    }
    return n;
}

cudaError_t launch_walks(const WalkLaunch& L, const DevProblem* d_probs, int n_probs, unsigned long long total,
                         DevCounters* d_counters, cudaStream_t stream, int* blocks_used, const DevProblem* host_prob,
                         DevCounters* zero_counters) {
    if (n_probs < 1 || n_probs > kMaxProblems) return cudaErrorInvalidValue;
    if (host_prob ? (n_probs != 1 || d_probs) : !d_probs) return cudaErrorInvalidValue;
    if (total == 0) {
        if (blocks_used) *blocks_used = 0;
        if (zero_counters) return cudaMemsetAsync(zero_counters, 0, sizeof(DevCounters), stream);
        return cudaSuccess;
    }
    const int bs = L.block_size;
    if (L.star && n_probs != 1) return cudaErrorInvalidValue;
    int per_sm = L.blocks_per_sm > 0 ? L.blocks_per_sm
                                     : walk_max_blocks_per_sm(L.dim, bs, L.traversal, L.star, L.cones, L.data);
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)per_sm * L.n_sm;
    const long long need = (long long)((total + bs - 1) / bs);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    if (blocks_used) *blocks_used = (int)blocks;
    if (bs % 32 != 0) return cudaErrorInvalidValue;
    const size_t smem = walk_smem_bytes(n_probs, bs, L.traversal, L.dim, L.star);
    DevProblem P1;
    if (host_prob) P1 = *host_prob;
    else memset(&P1, 0, sizeof(P1));
    auto go = [&](auto kernel) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kernel<<<(int)blocks, bs, smem, stream>>>(d_probs, n_probs, total, d_counters, zero_counters, P1);
        return cudaGetLastError();
    };
    if (L.star) {
        const bool wide = L.traversal == 2 || L.traversal == 3;
        if (L.data) {   // normal cones only prune; the data instantiation runs without them
            if (wide) return L.dim == 2 ? go(walk_kernel<2, true, true, false, true>)
                                        : go(walk_kernel<3, true, true, false, true>);
            return L.dim == 2 ? go(walk_kernel<2, false, true, false, true>) : go(walk_kernel<3, false, true, false, true>);
        }
        if (L.cones) {
            if (wide) return L.dim == 2 ? go(walk_kernel<2, true, true, true>) : go(walk_kernel<3, true, true, true>);
            return L.dim == 2 ? go(walk_kernel<2, false, true, true>) : go(walk_kernel<3, false, true, true>);
        }
        if (wide) return L.dim == 2 ? go(walk_kernel<2, true, true>) : go(walk_kernel<3, true, true>);
        return L.dim == 2 ? go(walk_kernel<2, false, true>) : go(walk_kernel<3, false, true>);
    }
    if (L.traversal == 2 || L.traversal == 3) return L.dim == 2 ? go(walk_kernel<2, true>) : go(walk_kernel<3, true>);
    return L.dim == 2 ? go(walk_kernel<2, false>) : go(walk_kernel<3, false>);
}

}  // namespace dwos
