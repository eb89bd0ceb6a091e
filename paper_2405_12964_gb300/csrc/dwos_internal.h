// Host/device shared declarations of the library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/dwos.h"

namespace dwos {

// The reflecting Neumann part of a mixed boundary (walk on stars): its own
// BVH, its elements in compact numbering with their neighbours (for the
// silhouette test), and the map from the Dirichlet BVH's compact element
// numbering to the input numbering.
struct DevNeumann {
    const float4* nodes;        // binary BVH of the Neumann elements (layout of the main BVH)
    const float4* prims;
    const int* prim_elem;       // leaf -> Neumann element (compact)
    int n_internal, n_tree, n_big, pad;
    const int* elem;            // compact Neumann elements, dim vertex ids each
    const int* adj;             // per Neumann element and endpoint (2D) / edge ab, bc, ca (3D): the
                                // neighbour's vertex across it, -1 where the Neumann part ends
    const float* vert;          // current vertices
    const int* dmap;            // Dirichlet element (compact, the main BVH's numbering) -> input element
    const float4* q_start;      // per query point of the current call: normal out of the domain (xyz) and
                                // the Neumann element (compact, int bits in w) its walk starts on, -1 inside
    // silhouette candidates: the sites (element endpoint in 2D, edge in 3D) where the Neumann part
    // ends or does not run straight on (every site when its vertices move with the parameters),
    // grouped by element, with a binary BVH over the elements that have one
    const float4* sil_nodes;
    const float4* sil_prims;
    const int* sil_prim;        // leaf -> entry of sites
    const int* sites;           // 8 e + mask: compact Neumann element e, bit j for its endpoint / edge j
    int sil_n_internal, sil_n_tree, sil_n_big, n_sites;   // n_sites: entries of sites
    // normal cones of that tree (NULL: none): per internal node and per leaf an axis (xyz) and a
    // half-angle (w, radians; >= 3 for the whole sphere) covering the sites' normal pairs,
    // oriented consistently across each site (a site is a silhouette from x only where its two
    // normals n satisfy n . (x - p) with opposite signs)
    const float4* sil_cone_node;
    const float4* sil_cone_leaf;
    // the silhouette rule's collinear tolerance seen as an angle about the perpendicular: at most
    // cone_tol (distance + cone_lmax), cone_tol = 1e-4 / (the smallest segment length, 3D: triangle
    // height over a candidate edge), cone_lmax the largest element size
    float cone_tol, cone_lmax;
    // Neumann data du/dn (n out of the domain) per compact Neumann element; NULL: zero everywhere
    // (a reflecting boundary)
    const float* flux;
};

// Everything a walk needs about one problem.  Copied to the device (and, in
// the walk kernel, into shared memory) once per launch.
struct DevProblem {
    // BVH and mesh
    const float4* nodes;
    const float4* prims;
    const int* prim_elem;       // leaf (Morton order) -> input element id
    const int* elem;            // n_elem x dim vertex ids
    const float* g_vert;        // n_vert (mapped data)
    int root;
    int n_internal;
    int n_tree;                 // leaves in the LBVH
    int n_big;                  // outsized elements after them
    const int* leaf_parent;     // leaf -> parent node
    const float* node_cell;     // Morton cell per internal node
    float r_max;                // element radius bound for the cell test
    int traversal;              // 0 root-down, 1 climb from the hint leaf, 2 warp-wide over the 32-wide tree,
                                // 3 routed: no tree search if the binary root's child boxes are outside the
                                // bound, else warp-wide (per lane when many lanes need one in a step)
    const float* wnodes;        // 32-wide tree (SoA nodes), root first
    int n_wide;                 // its node count
    int data_kind;              // 0 mapped, 1 field
    int differential;
    float field[10];            // c0, c(3), Axx Ayy Azz Axy Axz Ayz
    float sqrt_sigma;
    float f;
    float eps;
    float h;
    float inv_h;
    int K;
    int max_steps;
    int dudn_mode;              // 0 backward difference (Eq. dudn_fd_estimate), 1 ball gradient (Eq. dudn_mc_estimate)
    uint32_t seed_lo, seed_hi;
    // work
    const float* xq;            // n_query x dim
    const int* valid;           // n_query inside flags, or null (no check)
    int walks;                  // walks per point
    int node_budget;            // node fetches one distance query may make (0: the tree's own bound)
    unsigned long long walk_id_base;
    unsigned long long work_begin;   // first global work index of this problem
    unsigned long long work_end;
    // outputs
    dwos_record* rec;           // one per walk (local index p*W + w)
    uint32_t* trace;            // (K+1) per walk or null
    dwos_walk_debug* dbg;       // one per walk or null
    float4* cv_sample;          // per walk: main walk's first-step point x1 and its source S0, or null
    float4* cv_end;             // per walk: main walk's last point (where it stopped), or null
    const float4* cv_elem;      // per element (q, t): surrogate grad u = q n + t for the nested walks' correction, or null
    const DevNeumann* neu;      // reflecting Neumann part (walk on stars), or null
};

// Control variate applied by the estimator kernels: u - grad(x0) . (x1 - x0)
// for walks whose main walk took its first step (cv_sample x is not NaN).
struct CvView {
    const float4* sample;       // per walk (x1, S0), NaN x when the walk did not move
    const float* grad;          // n_query x dim
    const float* xq;            // n_query x dim
    int dim;
    const float4* end;          // if set: use the whole walk's displacement x_end - x0 instead of x1 - x0
};

struct DevCounters {
    unsigned long long next_work;
    unsigned long long steps_main;
    unsigned long long steps_nested;
    unsigned long long capped;
    unsigned long long nodes;   // binary BVH node fetches
    unsigned long long prims;   // element distance tests
    unsigned long long wnodes;  // 32-wide node visits
    int error;                  // bit 0: traversal bound exceeded, bit 1: query outside Omega,
                                // bit 2: query point not finite
    int pad[1];
};

// BVH build (bvh.cu).  All pointers are device pointers; work on `stream`.
struct BvhBuffers {
    int dim = 0, n_elem = 0, n_internal = 0;
    bool cells_ok = false;        // node_cell / r_max describe the elements (false after a refit):
                                  // search order 1 needs them
    int n_tree = 0, n_big = 0;    // leaves in the LBVH, outsized elements kept out of it
    float4* nodes = nullptr;      // max(1, n_elem-1) nodes
    float4* prims = nullptr;      // n_elem prims
    int* prim_elem = nullptr;     // n_elem
    int* leaf_of_elem = nullptr;  // n_elem: element -> leaf
    // scratch
    unsigned int* keys = nullptr;
    unsigned int* keys_sorted = nullptr;
    int* vals = nullptr;
    int* vals_sorted = nullptr;
    int* leaf_parent = nullptr;
    int* node_parent = nullptr;
    int* node_child = nullptr;    // 2 per internal node
    int* counters = nullptr;
    int* node_count = nullptr;       // per internal node: leaves under it; then (second half) its first leaf
    float* node_cell = nullptr;      // Morton cell box per internal node
    float r_max = 0.0f;              // largest element half box diagonal (tree elements)
    unsigned int* bounds = nullptr;  // 2*dim ordered-uint scene bounds
    float* stats = nullptr;          // size statistics + outsized count
    void* sort_tmp = nullptr;
    size_t sort_tmp_bytes = 0;
    int capacity = 0;
    // 32-wide tree collapsed from the binary one (rebuilt with it), nodes in level order
    float* wnodes = nullptr;         // n_wide x WideLayout<dim>::kFloats
    int* wsrc = nullptr;             // per slot: (binary parent << 1 | side) of the child's box, -1 unused
    int n_wide = 0, wide_depth = 0, wide_cap = 0;
    bool wide_ok = false;            // the warp-wide search fits its stack on this tree
};

cudaError_t bvh_reserve(BvhBuffers& b, int dim, int n_elem);
void bvh_free(BvhBuffers& b);
cudaError_t bvh_build(BvhBuffers& b, int dim, const float* vert, const int* elem, int n_elem,
                      cudaStream_t stream);
// New boxes for moved vertices over the same elements and tree topology (binary
// and 32-wide): every box again bounds its subtree, so the exact searches of
// orders 0, 2 and 3 stay exact; no host synchronisation and no allocation.
// The Morton cells go stale (cells_ok = false).
cudaError_t bvh_refit(BvhBuffers& b, const float* vert, const int* elem, cudaStream_t stream);

// Batched queries through the BVH (bvh.cu).
cudaError_t launch_closest(const BvhBuffers& b, int n, const float* p, const int* hint_elem, float* dist,
                           int* elem_out, float* bary, int* err, DevCounters* counters, int traversal,
                           cudaStream_t stream);
// Inside flags by ray parity.  prev (optional): the points of the call that
// left `inside` as it is; a point equal to its prev entry bit for bit keeps its
// flag.  prev_out (optional, may equal prev): receives the points.
cudaError_t launch_inside(const BvhBuffers& b, int n, const float* p, int* inside, cudaStream_t stream,
                          const float* prev = nullptr, float* prev_out = nullptr);
cudaError_t launch_philox(int n, const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out,
                          cudaStream_t stream);
cudaError_t launch_apply_params(const float* vert_ref, const float* jac, const float* theta, float* vert,
                                int n_rows, int n_param, cudaStream_t stream);

// Walk kernel (walk.cu).
struct WalkLaunch {
    int dim;
    int block_size;
    int blocks_per_sm;
    int n_sm;
    int traversal = 0;          // 2, 3: warp-wide search (every problem of the launch has wide_ok)
    bool star = false;          // walk on stars (one problem with a Neumann part)
    bool cones = false;         // walk on stars whose silhouette tree has normal cones
    bool data = false;          // walk on stars with Neumann data (runs without the cones)
};
// The problems come from the device table d_probs, or (one problem, d_probs
// NULL) by value from host_prob.  zero_counters, when given, is zeroed by the
// launch for the next one (the launch itself uses d_counters).
cudaError_t launch_walks(const WalkLaunch& L, const DevProblem* d_probs, int n_probs,
                         unsigned long long total_work, DevCounters* d_counters, cudaStream_t stream,
                         int* blocks_used, const DevProblem* host_prob = nullptr,
                         DevCounters* zero_counters = nullptr);
int walk_max_blocks_per_sm(int dim, int block_size, int traversal = 0, bool star = false, bool cones = false,
                           bool data = false);
// Query points on the Neumann part: per point the closest Neumann element if it
// lies within tol of it (q_start w = its compact index, xyz = its unit normal,
// not yet oriented) and the point 1e-3 of the element's size behind its centre
// along that normal (behind, dim floats); -1 and the point itself otherwise.
cudaError_t launch_neumann_start(int dim, int n, const float* xq, const DevNeumann& N, float tol,
                                 float4* q_start, float* behind, cudaStream_t stream);
// Orients each start normal out of the domain (flipped where the point behind the
// centre is outside) and marks the point valid (valid may be null).
cudaError_t launch_neumann_orient(int n, const int* behind_inside, float4* q_start, int* valid,
                                  cudaStream_t stream);
// The walk step's ball weights (source factor for uniform u, recursive weight) and the
// K0 of the 2D source weight, evaluated as the walk kernel evaluates them (walk.cu).
cudaError_t launch_ball_weights(int dim, float k, int n, const float* d, const float* u, float* src, float* alpha,
                                cudaStream_t stream);
cudaError_t launch_bessel_k(int order, int n, const float* x, float* out, cudaStream_t stream);
cudaError_t launch_star_weight(int dim, float k, int n, const float* t, const float* R, float* out, cudaStream_t stream);

// Estimator reductions (estimators.cu).
// mean / SE of the first `used` (0: all W) walks of each point
cudaError_t launch_reduce_u(const dwos_record* rec, int n_points, int W, double* mean, double* se,
                            cudaStream_t stream, const CvView* cv = nullptr, int used = 0);
// the control-variate network's training rows from thinned walks (see dwos_cv_training_set)
cudaError_t launch_cv_rows(const float4* samples, const dwos_walk_debug* dbg, long long n_rows, long long off,
                           long long stride, float h, float q_weight, float* x, float* t, float* m, double* acc,
                           cudaStream_t stream);
// per-walk training samples: s.w <- u - s.w (the estimate of u at x1) where x1 exists
cudaError_t launch_pack_samples(const dwos_record* rec, float4* samples, long long n, cudaStream_t stream);
cudaError_t launch_reduce_udot(const dwos_record* rec, const int* elem, const float* jac, const float* dg,
                               int dim, int n_param, int n_points, int W, double* mean, double* se,
                               cudaStream_t stream);
// mode 0: VJP weights w_p / W;  1: U-statistic L2 weights in batches of B;  2: correlated
// product (umean = mean u of all W walks);  3: uncorrelated product (umean = mean u of the
// first W/2 walks, weights on the other W/2).
// active (optional, one byte per vertex): scatter only into vertices whose flag is set
// (the others have zero Jacobian and dg rows, so they cannot reach the parameter gradient).
cudaError_t launch_scatter(const dwos_record* rec, const int* elem, int dim, int n_points, int W, int B,
                           int mode, const float* cot_or_uref, double* acc_vert, double* acc_g,
                           cudaStream_t stream, const CvView* cv = nullptr, const double* umean = nullptr,
                           const float* pweight = nullptr, const unsigned char* active = nullptr,
                           double* usum = nullptr, double* zero_out = nullptr, int n_zero = 0);
// usum (optional, n_points, zeroed by the caller): receives the per-point sums
// of u (FP64 over walks).  zero_out (optional): n_zero doubles zeroed by the
// launch, for a later kernel that accumulates into them.
// out[v] = 1 if vertex v has a nonzero entry in its Jacobian rows (dim x n_param) or its dg row.
cudaError_t launch_vertex_active(const float* jac, const float* dg, int n_vert, int dim, int n_param,
                                 unsigned char* out, cudaStream_t stream);
cudaError_t launch_gemv(const float* jac, const float* dg, const double* acc_vert, const double* acc_g,
                        int n_vert, int dim, int n_param, double* grad, cudaStream_t stream);
// 1/2 sum_p w_p (mean_p - uref_p)^2 with w = pweight (or 1)
cudaError_t launch_loss(const double* mean, const float* uref, int n_points, double* loss,
                        cudaStream_t stream, const float* pweight = nullptr, double scale = 1.0,
                        double* mean_out = nullptr);

}  // namespace dwos
