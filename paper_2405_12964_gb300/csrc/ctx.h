// Private: the context object behind the opaque dwos_ctx handle.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "dwos_internal.h"

struct dwos_ctx {
    int device = 0;
    int n_sm = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    dwos_options opt{};
    int node_budget = 0;         // node fetches per distance query (0: the tree's own bound)


    // boundary
    int dim = 0, n_vert = 0, n_elem = 0, n_param = 0;
    float* vert_ref = nullptr;   // n_vert*dim
    float* vert = nullptr;       // current vertices
    int* elem = nullptr;
    float* jac = nullptr;        // n_vert*dim*n_param (or null)
    float* theta = nullptr;      // n_param
    float* g_vert = nullptr;     // n_vert
    float* dg_vert = nullptr;    // n_vert*n_param or null
    unsigned char* vert_active = nullptr; size_t vert_active_cap = 0;   // vertex has a nonzero Jacobian / dg row
    bool active_stale = true;    // vert_active must be recomputed (Jacobian or data changed)
    int data_kind = 0;
    double field[10] = {0};
    float sigma = 0.0f, f = 0.0f;
    dwos::BvhBuffers bvh;        // over every element, or over the Dirichlet part when there is a Neumann part
    int refits = 0;              // parameter updates applied by refitting since the last full build
    bool have_boundary = false;
    // Neumann part (walk on stars); n_neumann = 0 when every element is Dirichlet
    int n_neumann = 0;
    int* elem_d = nullptr;       // compact Dirichlet elements (the main BVH's numbering)
    int* elem_n = nullptr;       // compact Neumann elements
    int* dmap = nullptr;         // compact Dirichlet element -> input element
    int* nadj = nullptr;         // per Neumann element and endpoint / edge: the neighbour's vertex, -1 open
    dwos::BvhBuffers bvh_n;      // over the Neumann part
    int n_sites = 0;             // elements with silhouette candidates (DevNeumann::sites)
    int* sites = nullptr;
    int* elem_s = nullptr;       // per entry of sites its element's vertices (what their BVH bounds)
    dwos::BvhBuffers bvh_s;      // over the silhouette candidates
    float4* sil_cones = nullptr; // their tree's normal cones: internal nodes, then leaves
    // host copies for the cones: compact Neumann elements, neighbours, site entries, vertices at
    // dwos_set_neumann, and whether a Neumann vertex moves with theta (then no cones)
    std::vector<int32_t> elem_n_h, nadj_h, sites_h;
    std::vector<float> vert_neu_h;
    bool neu_moving = false;
    float cone_tol = 1e30f, cone_lmax = 0.0f;               // DevNeumann::cone_tol, cone_lmax
    // Neumann data du/dn: per input element as given (empty: none), and per compact Neumann
    // element on the device (NULL when zero on the whole Neumann part); compact -> input element
    std::vector<float> neu_data_h;
    float* neu_data = nullptr;
    std::vector<int32_t> nmap_h;
    dwos::DevNeumann* d_neu = nullptr;
    dwos::DevNeumann neu_host{};                          // what d_neu holds
    float4* q_start = nullptr; size_t q_start_cap = 0;    // per query: start on the Neumann part
    float* behind = nullptr; size_t behind_cap = 0;       // per query: the orientation test point
    int* behind_in = nullptr; size_t behind_in_cap = 0;
    int* inside_tmp = nullptr; size_t inside_tmp_cap = 0;

    // workspaces (grow-only)
    dwos_record* rec = nullptr; size_t rec_cap = 0;
    float* xq = nullptr; size_t xq_cap = 0;           // host query points staged on the device
    const float* xq_in = nullptr;                         // the query points the last walks read
    float* xq_prev = nullptr; size_t xq_prev_cap = 0;     // the points whose inside flags `valid` holds
    int inside_cached = -1;                               // their count (-1: none, e.g. after a rebuild)
    int* valid = nullptr; size_t valid_cap = 0;
    float* wvec = nullptr; size_t wvec_cap = 0;           // cotangent / uref
    float* pw = nullptr; size_t pw_cap = 0;               // per-point quadrature weights
    double* out = nullptr; size_t out_cap = 0;            // reduced outputs
    double* acc_vert = nullptr; size_t acc_cap = 0;       // n_vert*dim + n_vert
    uint32_t* trace = nullptr; size_t trace_cap = 0;
    dwos_walk_debug* dbg = nullptr; size_t dbg_cap = 0;
    float* misc_f = nullptr; size_t misc_f_cap = 0;
    int* misc_i = nullptr; size_t misc_i_cap = 0;
    uint32_t* misc_u = nullptr; size_t misc_u_cap = 0;
    double* misc_d = nullptr; size_t misc_d_cap = 0;
    dwos::DevCounters* d_ctr = nullptr;   // two: the current launch's and the next one's (kept zero)
    int ctr_cur = 0;
    bool ctr_next_zero = true;
    int* d_err = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool timed = false;
    unsigned long long launches = 0;   // kernels launched by this context
    int last_blocks = 0;
};
