// Linear BVH over boundary elements, built on the device:
//   element boxes + scene bounds -> Morton codes -> radix sort (CUB) ->
//   binary radix tree (Karras, "Maximizing parallelism in the construction of
//   BVHs, octrees and k-d trees", HPG 2012) -> bottom-up box refit with
//   arrival counters -> leaf primitives written in Morton order -> 32-wide
//   tree collapsed from the binary one five levels at a time.
// Plus the batched closest-point, ray-parity inside test and Philox kernels.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <cstring>
#include <utility>
#include <vector>

#include "dwos_device.cuh"
#include "dwos_internal.h"

namespace dwos {

namespace {

__device__ __forceinline__ unsigned int float_to_ordered(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

template <int DIM>
__device__ __forceinline__ void elem_box(const float* vert, const int* elem, int e, float* lo, float* hi) {
#pragma unroll
    for (int k = 0; k < DIM; ++k) { lo[k] = kInf; hi[k] = -kInf; }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const int v = elem[DIM * e + a];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const float x = vert[DIM * v + k];
            lo[k] = fminf(lo[k], x);
            hi[k] = fmaxf(hi[k], x);
        }
    }
}

template <int DIM>
__device__ __forceinline__ float elem_diag(const float* vert, const int* elem, int e) {
    float lo[DIM], hi[DIM];
    elem_box<DIM>(vert, elem, e, lo, hi);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) s += (hi[k] - lo[k]) * (hi[k] - lo[k]);
    return sqrtf(s);
}

// Sum of element box diagonals (stats[0]) for the mean size.
template <int DIM>
__global__ void size_kernel(const float* vert, const int* elem, int n, float* stats) {
    float s = 0.0f;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        s += elem_diag<DIM>(vert, elem, e);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(stats, s);
}

// Elements whose box diagonal exceeds kBigFactor x the mean: count (stats[1]).
constexpr float kBigFactor = 16.0f;

// Also the largest half box diagonal over the elements that stay in the tree
// (stats_i[1]) and over all elements (stats_i[2]), as float bits.
template <int DIM>
__global__ void count_big_kernel(const float* vert, const int* elem, int n, float* stats, int* count) {
    const float thr = kBigFactor * stats[0] / (float)n;
    int c = 0;
    float r_small = 0.0f, r_all = 0.0f;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const float dgn = elem_diag<DIM>(vert, elem, e);
        const bool big = dgn > thr;
        c += big ? 1 : 0;
        r_all = fmaxf(r_all, 0.5f * dgn);
        if (!big) r_small = fmaxf(r_small, 0.5f * dgn);
    }
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        r_small = fmaxf(r_small, __shfl_xor_sync(0xffffffffu, r_small, o));
        r_all = fmaxf(r_all, __shfl_xor_sync(0xffffffffu, r_all, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (c) atomicAdd(count, c);
        atomicMax(count + 1, __float_as_int(r_small));   // non-negative floats order as ints
        atomicMax(count + 2, __float_as_int(r_all));
    }
}

// Scene bounds of the tree elements' centroids (ordered-uint encoding).
template <int DIM>
__global__ void bounds_kernel(const float* vert, const int* elem, int n, const float* stats, int split,
                              unsigned int* bounds) {
    const float thr = split ? kBigFactor * stats[0] / (float)n : kInf;
    float lo[DIM], hi[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) { lo[k] = kInf; hi[k] = -kInf; }
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        float l[DIM], h[DIM];
        elem_box<DIM>(vert, elem, e, l, h);
        float d2 = 0.0f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) d2 += (h[k] - l[k]) * (h[k] - l[k]);
        if (sqrtf(d2) > thr) continue;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const float c = 0.5f * (l[k] + h[k]);
            lo[k] = fminf(lo[k], c);
            hi[k] = fmaxf(hi[k], c);
        }
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            atomicMin(bounds + k, float_to_ordered(lo[k]));
            atomicMax(bounds + DIM + k, float_to_ordered(hi[k]));
        }
    }
}

__device__ __forceinline__ unsigned int spread2(unsigned int x) {   // 16 bits -> even bits
    x &= 0xffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}
__device__ __forceinline__ unsigned int spread3(unsigned int x) {   // 10 bits -> every third bit
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// 30-bit Morton code of the centroid (15 bits per axis in 2D, 10 in 3D);
// outsized elements get 0xFFFFFFFF so that the sort puts them last, in index order.
template <int DIM>
__global__ void morton_kernel(const float* vert, const int* elem, int n, const unsigned int* bounds,
                              const float* stats, int split, unsigned int* keys, int* vals) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    vals[e] = e;
    float l[DIM], h[DIM];
    elem_box<DIM>(vert, elem, e, l, h);
    float d2 = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) d2 += (h[k] - l[k]) * (h[k] - l[k]);
    if (split && sqrtf(d2) > kBigFactor * stats[0] / (float)n) { keys[e] = 0xFFFFFFFFu; return; }
    unsigned int q[DIM];
    const float levels = DIM == 2 ? 32767.0f : 1023.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const float lo = ordered_to_float(bounds[k]);
        const float hi = ordered_to_float(bounds[DIM + k]);
        const float ext = hi - lo;
        float t = ext > 0.0f ? (0.5f * (l[k] + h[k]) - lo) / ext : 0.5f;
        t = fminf(fmaxf(t, 0.0f), 1.0f);
        q[k] = (unsigned int)(t * levels + 0.5f);
    }
    keys[e] = DIM == 2 ? (spread2(q[0]) | (spread2(q[1]) << 1))
                       : (spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2));
}

// Length of the common prefix of keys i and j, with the index as tie-breaker;
// -1 outside [0, n).
__device__ __forceinline__ int delta(const unsigned int* k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const unsigned int a = k[i], b = k[j];
    if (a == b) return 32 + __clz((unsigned int)(i ^ j));
    return __clz(a ^ b);
}

// Box of centroids admitted by a Morton prefix: the top p bits of the 30-bit
// code fix the top bits of each axis; q = floor(t * levels + 0.5) lies in
// [q_lo, q_hi] iff t lies in [(q_lo - 0.5)/levels, (q_hi + 0.5)/levels).
template <int DIM>
__device__ void morton_cell(unsigned int key, int p, const unsigned int* bounds, float* cell) {
    const int B = DIM == 2 ? 15 : 10;
    const float levels = DIM == 2 ? 32767.0f : 1023.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int n_a = 0;
        for (int b = 29; b >= 30 - p; --b) n_a += (b % DIM == a) ? 1 : 0;
        unsigned int q = 0;
        for (int k = 0; k < B; ++k) q |= ((key >> (DIM * k + a)) & 1u) << k;
        const unsigned int q_lo = n_a > 0 ? ((q >> (B - n_a)) << (B - n_a)) : 0u;
        const unsigned int q_hi = q_lo + (1u << (B - n_a)) - 1u;
        const float lo = ordered_to_float(bounds[a]);
        const float ext = ordered_to_float(bounds[DIM + a]) - lo;
        if (!(ext > 0.0f)) {              // flat axis: the code does not separate along it
            cell[a] = -kInf;
            cell[DIM + a] = kInf;
            continue;
        }
        cell[a] = lo + (((float)q_lo - 0.5f) / levels) * ext;
        cell[DIM + a] = lo + (((float)q_hi + 0.5f) / levels) * ext;
    }
}

template <int DIM>
__global__ void radix_tree_kernel(const unsigned int* keys, int n, int* node_child, int* node_parent,
                                  int* leaf_parent, const unsigned int* bounds, float* node_cell, int* node_count,
                                  int* node_first) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int dir = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(keys, n, i, i - dir);
    int lmax = 2;
    while (delta(keys, n, i, i + lmax * dir) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, n, i, i + (l + t) * dir) > dmin) l += t;
    const int j = i + l * dir;
    const int dnode = delta(keys, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(keys, n, i, i + (s + t) * dir) > dnode) s += t;
    } while (t > 1);
    const int split = i + s * dir + min(dir, 0);
    const int first = min(i, j), last = max(i, j);
    node_count[i] = last - first + 1;               // leaves under node i: first .. last
    node_first[i] = first;
    int left, right;
    if (first == split) { left = ~split; leaf_parent[split] = i; }
    else { left = split; node_parent[split] = i; }
    if (last == split + 1) { right = ~(split + 1); leaf_parent[split + 1] = i; }
    else { right = split + 1; node_parent[split + 1] = i; }
    node_child[2 * i] = left;
    node_child[2 * i + 1] = right;
    if (i == 0) node_parent[0] = -1;
    // keys of this node's range share dnode leading bits (>= 32: all equal)
    const int p = dnode >= 32 ? 30 : dnode - 2;
    morton_cell<DIM>(keys[i], p, bounds, node_cell + 2 * DIM * i);
}

template <int DIM>
__device__ __forceinline__ void write_child_box(float4* nodes, int node, int slot, const float* lo,
                                                const float* hi) {
    float* f = reinterpret_cast<float*>(nodes + BvhLayout<DIM>::kNodeF4 * node);
    if (DIM == 2) {
        float* b = f + 4 * slot;
        b[0] = lo[0]; b[1] = lo[1]; b[2] = hi[0]; b[3] = hi[1];
    } else {
        float* b = f + 6 * slot;
        b[0] = lo[0]; b[1] = lo[1]; b[2] = lo[2]; b[3] = hi[0]; b[4] = hi[1]; b[5] = hi[2];
    }
}

template <int DIM>
__global__ void refit_kernel(const float* vert, const int* elem, const int* sorted_elem, int n,
                             const int* node_child, const int* node_parent, const int* leaf_parent,
                             int* counters, float4* nodes) {
    const int leaf = blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= n) return;
    float lo[DIM], hi[DIM];
    elem_box<DIM>(vert, elem, sorted_elem[leaf], lo, hi);
    int child = ~leaf;
    int node = leaf_parent[leaf];
    while (node >= 0) {
        const int slot = (node_child[2 * node] == child) ? 0 : 1;
        write_child_box<DIM>(nodes, node, slot, lo, hi);
        __threadfence();                                   // publish this child's box
        if (atomicAdd(counters + node, 1) == 0) return;    // the sibling finishes this node
        __threadfence();
        // second arrival: the node's bounds are the union of both child slots (read through L2)
        const volatile float* f = reinterpret_cast<const volatile float*>(nodes + BvhLayout<DIM>::kNodeF4 * node);
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            float a_lo, a_hi, b_lo, b_hi;
            if (DIM == 2) { a_lo = f[k]; a_hi = f[2 + k]; b_lo = f[4 + k]; b_hi = f[6 + k]; }
            else { a_lo = f[k]; a_hi = f[3 + k]; b_lo = f[6 + k]; b_hi = f[9 + k]; }
            lo[k] = fminf(a_lo, b_lo);
            hi[k] = fmaxf(a_hi, b_hi);
        }
        child = node;
        node = node_parent[node];
    }
}

template <int DIM>
__global__ void finalize_kernel(const float* vert, const int* elem, const int* sorted_elem, int n,
                                const int* node_child, const int* node_parent, int n_internal,
                                float4* nodes, float4* prims, int* prim_elem, int* leaf_of_elem) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_internal && node_child) {
        float4* m = nodes + BvhLayout<DIM>::kNodeF4 * i + (BvhLayout<DIM>::kNodeF4 - 1);
        *m = make_float4(__int_as_float(node_child[2 * i]), __int_as_float(node_child[2 * i + 1]),
                         __int_as_float(node_parent[i]), 0.0f);
    }
    if (i < n) {
        const int e = sorted_elem[i];
        prim_elem[i] = e;
        leaf_of_elem[e] = i;
        if (DIM == 2) {
            const int a = elem[2 * e], b = elem[2 * e + 1];
            prims[i] = make_float4(vert[2 * a], vert[2 * a + 1], vert[2 * b], vert[2 * b + 1]);
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int v = elem[3 * e + c];
                prims[3 * i + c] = make_float4(vert[3 * v], vert[3 * v + 1], vert[3 * v + 2], 0.0f);
            }
        }
    }
}

// One tree element: a single node whose right child is empty.
template <int DIM>
__global__ void single_leaf_kernel(const float* vert, const int* elem, const int* sorted_elem, float4* nodes,
                                   int* leaf_parent, float* node_cell) {
    leaf_parent[0] = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) { node_cell[k] = -kInf; node_cell[DIM + k] = kInf; }
    float lo[DIM], hi[DIM], elo[DIM], ehi[DIM];
    elem_box<DIM>(vert, elem, sorted_elem[0], lo, hi);
#pragma unroll
    for (int k = 0; k < DIM; ++k) { elo[k] = kInf; ehi[k] = -kInf; }
    write_child_box<DIM>(nodes, 0, 0, lo, hi);
    write_child_box<DIM>(nodes, 0, 1, elo, ehi);
    nodes[BvhLayout<DIM>::kNodeF4 - 1] =
        make_float4(__int_as_float(~0), __int_as_float(kEmptyChild), __int_as_float(-1), 0.0f);
}

// ---- 32-wide tree -----------------------------------------------------------
// Built top-down, one level per launch.  A wide node starts from its binary
// root's two children; it first opens, largest first, the inner children with
// more than 32 leaves (they cannot become one leaf-level node), then absorbs
// whole inner children that still fit as their leaves, largest first.  Its
// remaining inner children become the next level's wide nodes.  (Opening
// every child by size alone cuts small subtrees into pieces, each a nearly
// empty wide node: 37 % of the slots used on a 32 k-element test set against
// 71 % with this rule.)

// Frontier of each wide node of this level (in order), and its inner-child count.
__global__ void wide_level_kernel(const int* node_child, const int* node_count, const int* node_first,
                                  const int* leaf_parent, const int* roots, int m, int* fr_code, int* fr_src,
                                  int* n_inner) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= m) return;
    const int r = roots[w];
    int code[kWide], src[kWide];
    int cnt = 0;
    for (int side = 0; side < 2; ++side) {
        code[cnt] = node_child[2 * r + side];
        src[cnt] = (r << 1) | side;
        ++cnt;
    }
    auto leaves = [&](int c) { return c >= 0 ? node_count[c] : 1; };
    while (cnt < kWide) {                      // open the largest child with more than 32 leaves
        int pick = -1, best = kWide;
        for (int i = 0; i < cnt; ++i)
            if (code[i] >= 0 && leaves(code[i]) > best) { best = leaves(code[i]); pick = i; }
        if (pick < 0) break;
        const int c = code[pick];
        for (int i = cnt; i > pick + 1; --i) { code[i] = code[i - 1]; src[i] = src[i - 1]; }
        for (int side = 0; side < 2; ++side) {
            code[pick + side] = node_child[2 * c + side];
            src[pick + side] = (c << 1) | side;
        }
        ++cnt;
    }
    while (cnt < kWide) {                      // absorb the largest inner child that fits
        const int room = kWide - cnt + 1;
        int pick = -1, best = 0;
        for (int i = 0; i < cnt; ++i)
            if (code[i] >= 0 && leaves(code[i]) <= room && leaves(code[i]) > best) { best = leaves(code[i]); pick = i; }
        if (pick < 0) break;
        const int c = code[pick], k = node_count[c], f = node_first[c];
        for (int i = cnt - 1; i > pick; --i) { code[i + k - 1] = code[i]; src[i + k - 1] = src[i]; }
        for (int t = 0; t < k; ++t) {
            const int leaf = f + t, par = leaf_parent[leaf];
            code[pick + t] = ~leaf;
            src[pick + t] = (par << 1) | (node_child[2 * par] == ~leaf ? 0 : 1);
        }
        cnt += k - 1;
    }
    int inner = 0;
    for (int i = 0; i < kWide; ++i) {
        const bool used = i < cnt;
        fr_code[kWide * w + i] = used ? code[i] : kEmptyChild;
        fr_src[kWide * w + i] = used ? src[i] : -1;
        inner += (used && code[i] >= 0) ? 1 : 0;
    }
    n_inner[w] = inner;
}

// Wide-node codes of the inner children (the next level, numbered after
// next_base in order) and the next level's binary roots.
__global__ void wide_assign_kernel(const int* fr_code, const int* fr_src, const int* offset, int m, int next_base,
                                   int* wcode, int* wsrc, int* next_roots) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= m) return;
    int k = offset[w];
    for (int i = 0; i < kWide; ++i) {
        const int c = fr_code[kWide * w + i];
        wsrc[kWide * w + i] = fr_src[kWide * w + i];
        if (c >= 0 && c != kEmptyChild) {
            next_roots[k] = c;
            wcode[kWide * w + i] = next_base + k;
            ++k;
        } else {
            wcode[kWide * w + i] = c;
        }
    }
}

// Child boxes gathered from the binary tree (its refit already ran) and codes.
template <int DIM>
__global__ void wide_refit_kernel(const float4* nodes, const float4* prims, const int* wsrc, const int* wcode,
                                  int n_wide, float* wnodes) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_wide * kWide) return;
    const int w = t / kWide, j = t % kWide;
    float* f = wnodes + (size_t)w * WideLayout<DIM>::kFloats;
    const int src = wsrc[t];
    float lo[DIM], hi[DIM];
    if (src < 0) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) { lo[k] = kInf; hi[k] = -kInf; }
    } else {
        const float* b = reinterpret_cast<const float*>(nodes + BvhLayout<DIM>::kNodeF4 * (src >> 1)) +
                         (DIM == 2 ? 4 : 6) * (src & 1);
#pragma unroll
        for (int k = 0; k < DIM; ++k) { lo[k] = b[k]; hi[k] = b[DIM + k]; }
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) { f[k * kWide + j] = lo[k]; f[(DIM + k) * kWide + j] = hi[k]; }
    const int code = wcode[t];
    f[2 * DIM * kWide + j] = __int_as_float(code);
    // a leaf child's vertices (the element in Morton order), zeros otherwise
    float v[DIM * DIM];
#pragma unroll
    for (int k = 0; k < DIM * DIM; ++k) v[k] = 0.0f;
    if (code < 0) {
        const int p = ~code;
        if constexpr (DIM == 2) {
            const float4 sgm = prims[p];
            v[0] = sgm.x; v[1] = sgm.y; v[2] = sgm.z; v[3] = sgm.w;
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float4 a = prims[3 * p + c];
                v[3 * c] = a.x; v[3 * c + 1] = a.y; v[3 * c + 2] = a.z;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < DIM * DIM; ++k) f[WideLayout<DIM>::kVtx + k * kWide + j] = v[k];
}

// ---- queries --------------------------------------------------------------
template <int DIM>
__global__ void closest_kernel(BvhView bvh, const int* prim_elem, const int* leaf_of_elem, int n, const float* p,
                               const int* hint_elem, float* dist, int* elem_out, float* bary, int* err,
                               DevCounters* ctr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float q[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) q[k] = p[DIM * i + k];
    float best2 = kInf;
    int best = -1;
    if (hint_elem) {   // seed with the caller's element, as a walk seeds with its previous hit
        const int h = hint_elem[i];
        if (h >= 0 && h < bvh.n_tree + bvh.n_big) {
            best = leaf_of_elem[h];
            best2 = prim_dist2<DIM>(bvh.prims, best, q);
        }
    }
    unsigned nn = 0, np = 0;
    if (!closest_leaf<DIM>(bvh, q, best2, best, nn, np)) atomicOr(err, 1);
    if (ctr) {
        atomicAdd(&ctr->nodes, (unsigned long long)nn);
        atomicAdd(&ctr->prims, (unsigned long long)np);
    }
    float w1 = 0.0f, w2 = 0.0f;
    if (best >= 0) {
        if (DIM == 2) {
            const float4 s = bvh.prims[best];
            best2 = seg_closest(q, s.x, s.y, s.z, s.w, w1);
        } else {
            const float4 a = bvh.prims[3 * best], b = bvh.prims[3 * best + 1], c = bvh.prims[3 * best + 2];
            best2 = tri_closest(q, make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z),
                                make_float3(c.x, c.y, c.z), w1, w2);
        }
    }
    dist[i] = sqrtf(best2);
    elem_out[i] = best >= 0 ? prim_elem[best] : -1;
    bary[2 * i] = w1;
    bary[2 * i + 1] = w2;
}

// The same query with the warp-wide search of the 32-wide tree: all lanes of a
// block take part (a lane past n only helps), so there is no early return.
template <int DIM>
__global__ void closest_wide_kernel(BvhView bvh, WideView wv, const int* prim_elem, const int* leaf_of_elem, int n,
                                    const float* p, const int* hint_elem, float* dist, int* elem_out, float* bary,
                                    int* err, DevCounters* ctr) {
    extern __shared__ float2 wide_stack[];
    float2* stk = wide_stack + (size_t)(threadIdx.x >> 5) * kWideStack;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = i < n;
    float q[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) q[k] = act ? p[DIM * i + k] : 0.0f;
    float best2 = kInf;
    int best = -1;
    unsigned nn = 0, np = 0;
    if (act) {
        if (hint_elem) {
            const int h = hint_elem[i];
            if (h >= 0 && h < bvh.n_tree + bvh.n_big) {
                best = leaf_of_elem[h];
                best2 = prim_dist2<DIM>(bvh.prims, best, q);
            }
        }
        big_closest<DIM>(bvh.prims, bvh.n_tree, bvh.n_big, q, best2, best, np);
    }
    const int e = wide_closest<DIM>(wv, __ballot_sync(kWarpAll, act), q, best2, best, stk, nn, np);
    if (e) atomicOr(err, 1);
    if (ctr) {
        atomicAdd(&ctr->wnodes, (unsigned long long)nn);
        atomicAdd(&ctr->prims, (unsigned long long)np);
    }
    if (!act) return;
    float w1 = 0.0f, w2 = 0.0f;
    if (best >= 0) {
        if (DIM == 2) {
            const float4 s = bvh.prims[best];
            best2 = seg_closest(q, s.x, s.y, s.z, s.w, w1);
        } else {
            const float4 a = bvh.prims[3 * best], b = bvh.prims[3 * best + 1], c = bvh.prims[3 * best + 2];
            best2 = tri_closest(q, make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z),
                                make_float3(c.x, c.y, c.z), w1, w2);
        }
    }
    dist[i] = sqrtf(best2);
    elem_out[i] = best >= 0 ? prim_elem[best] : -1;
    bary[2 * i] = w1;
    bary[2 * i + 1] = w2;
}

// Inside test by ray parity along a fixed generic direction.  The ray from
// each point is cut into 32 sub-intervals [t_s, t_s+1) up to the far corner of
// the scene box; lane s of the point's warp counts the crossings in its
// interval with an any-order stackless traversal (pruning boxes its interval
// misses) plus the outsized elements, and the warp sums the counts.
template <int DIM>
__device__ __forceinline__ bool seg_hits_box(const float* o, const float* inv, float ta, float tb, const float* lo,
                                             const float* hi) {
    float t0 = ta, t1 = tb;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const float a = (lo[k] - o[k]) * inv[k], b = (hi[k] - o[k]) * inv[k];
        t0 = fmaxf(t0, fminf(a, b));
        t1 = fminf(t1, fmaxf(a, b));
    }
    // a prefilter only: a ray through a box corner (a shared vertex) must not be
    // rejected by rounding, so the overlap test allows a small relative slack
    return t0 <= t1 + 1e-5f * fmaxf(1.0f, fabsf(t1));
}

// Ray parameter of the crossing with leaf p, or -1.  Watertight: a crossing
// through a vertex or edge shared by two elements is counted exactly once.
//  2D: crossing-number rule; each vertex's side of the ray's line is computed
//      from that vertex alone, so both segments sharing it agree.
//  3D: vertices are projected on the plane orthogonal to the ray (per-vertex
//      arithmetic, identical in every triangle); the 2D edge functions are
//      evaluated without contraction, so the two triangles of a shared edge get
//      exactly opposite values, and a zero value is broken by the edge's
//      direction, which the two triangles also see reversed.
struct RayFrame {
    float dir[3];
    float e1[3], e2[3];   // 3D: orthonormal basis of the plane orthogonal to dir
};

__device__ __forceinline__ float side2(const float* o, const float* dir, float vx, float vy) {
    return __fsub_rn(__fmul_rn(dir[0], __fsub_rn(vy, o[1])), __fmul_rn(dir[1], __fsub_rn(vx, o[0])));
}

__device__ __forceinline__ float edge_fn(float px, float py, float qx, float qy) {
    return __fsub_rn(__fmul_rn(px, qy), __fmul_rn(py, qx));
}

__device__ __forceinline__ bool edge_positive(float px, float py, float qx, float qy) {
    const float e = edge_fn(px, py, qx, qy);
    if (e != 0.0f) return e > 0.0f;
    return (qx > px) || (qx == px && qy > py);
}

__device__ __forceinline__ void project(const RayFrame& F, const float* o, float4 v, float& x, float& y, float& z) {
    const float dx = __fsub_rn(v.x, o[0]), dy = __fsub_rn(v.y, o[1]), dz = __fsub_rn(v.z, o[2]);
    x = __fadd_rn(__fadd_rn(__fmul_rn(dx, F.e1[0]), __fmul_rn(dy, F.e1[1])), __fmul_rn(dz, F.e1[2]));
    y = __fadd_rn(__fadd_rn(__fmul_rn(dx, F.e2[0]), __fmul_rn(dy, F.e2[1])), __fmul_rn(dz, F.e2[2]));
    z = __fadd_rn(__fadd_rn(__fmul_rn(dx, F.dir[0]), __fmul_rn(dy, F.dir[1])), __fmul_rn(dz, F.dir[2]));
}

template <int DIM>
__device__ __forceinline__ float ray_prim_t(const float4* prims, int p, const float* o, const RayFrame& F) {
    if (DIM == 2) {
        const float4 s = prims[p];
        const float sa = side2(o, F.dir, s.x, s.y), sb = side2(o, F.dir, s.z, s.w);
        if ((sa >= 0.0f) == (sb >= 0.0f)) return -1.0f;
        const float lam = sa / (sa - sb);
        const float ax = s.x - o[0], ay = s.y - o[1];
        return (ax + lam * (s.z - s.x)) * F.dir[0] + (ay + lam * (s.w - s.y)) * F.dir[1];
    } else {
        float ax, ay, az, bx, by, bz, cx, cy, cz;
        project(F, o, prims[3 * p], ax, ay, az);
        project(F, o, prims[3 * p + 1], bx, by, bz);
        project(F, o, prims[3 * p + 2], cx, cy, cz);
        // the projected origin is (0, 0): inside iff all edge functions share a sign
        const bool pa = edge_positive(bx, by, cx, cy);   // edge b -> c (weight of a)
        const bool pb = edge_positive(cx, cy, ax, ay);   // edge c -> a (weight of b)
        const bool pc = edge_positive(ax, ay, bx, by);   // edge a -> b (weight of c)
        if (!((pa && pb && pc) || (!pa && !pb && !pc))) return -1.0f;
        const float wa = edge_fn(bx, by, cx, cy), wb = edge_fn(cx, cy, ax, ay), wc = edge_fn(ax, ay, bx, by);
        const float den = wa + wb + wc;
        if (den == 0.0f) return -1.0f;
        return (wa * az + wb * bz + wc * cz) / den;
    }
}

template <int DIM>
__device__ __forceinline__ void prim_box(const float4* prims, int p, float* lo, float* hi) {
    if (DIM == 2) {
        const float4 s = prims[p];
        lo[0] = fminf(s.x, s.z); hi[0] = fmaxf(s.x, s.z);
        lo[1] = fminf(s.y, s.w); hi[1] = fmaxf(s.y, s.w);
    } else {
        const float4 a = prims[3 * p], b = prims[3 * p + 1], c = prims[3 * p + 2];
        lo[0] = fminf(a.x, fminf(b.x, c.x)); hi[0] = fmaxf(a.x, fmaxf(b.x, c.x));
        lo[1] = fminf(a.y, fminf(b.y, c.y)); hi[1] = fmaxf(a.y, fmaxf(b.y, c.y));
        lo[2] = fminf(a.z, fminf(b.z, c.z)); hi[2] = fmaxf(a.z, fmaxf(b.z, c.z));
    }
}

template <int DIM>
__global__ void inside_kernel(BvhView bvh, int n, const float* p, int* inside, const float* prev, float* prev_out) {
    const int pt = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (pt >= n) return;    // whole warps exit together
    float o[DIM], inv[DIM];
    RayFrame F;
    if (DIM == 2) {
        F.dir[0] = 0.8191520443f; F.dir[1] = 0.5735764364f; F.dir[2] = 0.0f;
    } else {
        // generic unit direction and an orthonormal basis of its normal plane
        F.dir[0] = 0.5144957554f; F.dir[1] = 0.6859943406f; F.dir[2] = 0.5144957554f;
        F.e1[0] = 0.7071067812f; F.e1[1] = 0.0f; F.e1[2] = -0.7071067812f;
        F.e2[0] = -0.4850712500f; F.e2[1] = 0.7276068751f; F.e2[2] = -0.4850712500f;
    }
    const float* dir = F.dir;
#pragma unroll
    for (int k = 0; k < DIM; ++k) { o[k] = p[DIM * pt + k]; inv[k] = 1.0f / dir[k]; }
    if (prev) {   // the same point as last time: its flag stands
        bool same = true;
#pragma unroll
        for (int k = 0; k < DIM; ++k) same = same && __float_as_uint(o[k]) == __float_as_uint(prev[DIM * pt + k]);
        if (same) return;
    }
    // scene box: the root's two children and the outsized elements
    float slo[DIM], shi[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) { slo[k] = o[k]; shi[k] = o[k]; }
    if (bvh.n_internal > 0) {
        float lo0[DIM], hi0[DIM], lo1[DIM], hi1[DIM];
        int c0, c1, parent;
        load_node<DIM>(bvh.nodes, bvh.root, lo0, hi0, lo1, hi1, c0, c1, parent);
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            slo[k] = fminf(slo[k], lo0[k]); shi[k] = fmaxf(shi[k], hi0[k]);
            if (c1 != kEmptyChild) { slo[k] = fminf(slo[k], lo1[k]); shi[k] = fmaxf(shi[k], hi1[k]); }
        }
    }
    for (int q = bvh.n_tree; q < bvh.n_tree + bvh.n_big; ++q) {
        float lo[DIM], hi[DIM];
        prim_box<DIM>(bvh.prims, q, lo, hi);
#pragma unroll
        for (int k = 0; k < DIM; ++k) { slo[k] = fminf(slo[k], lo[k]); shi[k] = fmaxf(shi[k], hi[k]); }
    }
    float tmax2 = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const float e = fmaxf(o[k] - slo[k], shi[k] - o[k]);
        tmax2 += e * e;
    }
    const float tmax = 1.001f * sqrtf(tmax2) + 1e-6f;
    const float ta = tmax * (float)lane / 32.0f;
    const float tb = lane == 31 ? 2.0f * tmax : tmax * (float)(lane + 1) / 32.0f;
    int count = 0;
    for (int q = bvh.n_tree; q < bvh.n_tree + bvh.n_big; ++q) {
        const float t = ray_prim_t<DIM>(bvh.prims, q, o, F);
        count += (t > 0.0f && t >= ta && t < tb) ? 1 : 0;
    }
    if (bvh.n_internal > 0) {
        int node = bvh.root, from = kFromParent;
        int budget = 3 * bvh.n_internal + 8;
        while (--budget >= 0) {
            float lo0[DIM], hi0[DIM], lo1[DIM], hi1[DIM];
            int c0, c1, parent;
            load_node<DIM>(bvh.nodes, node, lo0, hi0, lo1, hi1, c0, c1, parent);
            int state = from == kFromParent ? 0 : (from == c0 ? 1 : 2);
            int next = kFromParent;
            while (state < 2) {
                const int c = state == 0 ? c0 : c1;
                const bool hit = c != kEmptyChild &&
                                 (state == 0 ? seg_hits_box<DIM>(o, inv, ta, tb, lo0, hi0)
                                             : seg_hits_box<DIM>(o, inv, ta, tb, lo1, hi1));
                if (hit && c >= 0) { next = c; break; }
                if (hit) {
                    const float t = ray_prim_t<DIM>(bvh.prims, ~c, o, F);
                    count += (t > 0.0f && t >= ta && t < tb) ? 1 : 0;
                }
                ++state;
            }
            if (next != kFromParent) { from = kFromParent; node = next; continue; }
            if (parent < 0) break;
            from = node;
            node = parent;
        }
    }
    for (int off = 16; off > 0; off >>= 1) count += __shfl_xor_sync(0xffffffffu, count, off);
    if (lane == 0) {
        inside[pt] = count & 1;
        if (prev_out) {
#pragma unroll
            for (int k = 0; k < DIM; ++k) prev_out[DIM * pt + k] = o[k];
        }
    }
}

__global__ void philox_kernel(int n, const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const U4 r = philox(U4{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]}, k0, k1);
    out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
}

// v = v_ref + J theta, one thread per (vertex, coordinate) row.
__global__ void apply_params_kernel(const float* vert_ref, const float* jac, const float* theta, float* vert,
                                    int n_rows, int n_param) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    float s = vert_ref[r];
    const float* J = jac + (size_t)r * n_param;
    for (int j = 0; j < n_param; ++j) s = fmaf(J[j], theta[j], s);
    vert[r] = s;
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

cudaError_t bvh_reserve(BvhBuffers& b, int dim, int n_elem) {
    if (n_elem <= b.capacity && dim == b.dim) return cudaSuccess;
    bvh_free(b);
    const int n_int = n_elem > 1 ? n_elem - 1 : 1;
    const int nf4 = dim == 2 ? 3 : 4, pf4 = dim == 2 ? 1 : 3;
    cudaError_t e;
#define DW_TRY(x) do { e = (x); if (e != cudaSuccess) { bvh_free(b); return e; } } while (0)
    DW_TRY(cudaMalloc(&b.nodes, sizeof(float4) * nf4 * (size_t)n_int));
    DW_TRY(cudaMalloc(&b.prims, sizeof(float4) * pf4 * (size_t)n_elem));
    DW_TRY(cudaMalloc(&b.prim_elem, sizeof(int) * (size_t)n_elem));
    DW_TRY(cudaMalloc(&b.leaf_of_elem, sizeof(int) * (size_t)n_elem));
    DW_TRY(cudaMalloc(&b.keys, sizeof(unsigned int) * (size_t)n_elem));
    DW_TRY(cudaMalloc(&b.keys_sorted, sizeof(unsigned int) * (size_t)n_elem));
    DW_TRY(cudaMalloc(&b.vals, sizeof(int) * (size_t)n_elem));
    DW_TRY(cudaMalloc(&b.vals_sorted, sizeof(int) * (size_t)n_elem));
    DW_TRY(cudaMalloc(&b.leaf_parent, sizeof(int) * (size_t)n_elem));
    DW_TRY(cudaMalloc(&b.node_parent, sizeof(int) * (size_t)n_int));
    DW_TRY(cudaMalloc(&b.node_child, sizeof(int) * 2 * (size_t)n_int));
    DW_TRY(cudaMalloc(&b.counters, sizeof(int) * (size_t)n_int));
    DW_TRY(cudaMalloc(&b.node_count, sizeof(int) * 2 * (size_t)n_int));   // leaf counts, then first leaves
    DW_TRY(cudaMalloc(&b.node_cell, sizeof(float) * 2 * dim * (size_t)n_int));
    DW_TRY(cudaMalloc(&b.bounds, sizeof(unsigned int) * 6));
    DW_TRY(cudaMalloc(&b.stats, sizeof(float) * 2 + sizeof(int) * 4));
    size_t tmp = 0;
    DW_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp, b.keys, b.keys_sorted, b.vals, b.vals_sorted, n_elem));
    DW_TRY(cudaMalloc(&b.sort_tmp, tmp));
#undef DW_TRY
    b.sort_tmp_bytes = tmp;
    b.capacity = n_elem;
    b.dim = dim;
    return cudaSuccess;
}

void bvh_free(BvhBuffers& b) {
    cudaFree(b.nodes); cudaFree(b.prims); cudaFree(b.prim_elem); cudaFree(b.leaf_of_elem); cudaFree(b.keys); cudaFree(b.keys_sorted);
    cudaFree(b.vals); cudaFree(b.vals_sorted); cudaFree(b.leaf_parent); cudaFree(b.node_parent);
    cudaFree(b.node_child); cudaFree(b.counters); cudaFree(b.bounds); cudaFree(b.stats); cudaFree(b.node_cell);
    cudaFree(b.sort_tmp);
    cudaFree(b.wnodes); cudaFree(b.wsrc); cudaFree(b.node_count);
    b = BvhBuffers();
}

constexpr int kMaxBig = 64;

// Collapse the binary tree (n_internal >= 1 nodes, boxes refit) into the
// 32-wide tree, level by level (one host synchronisation per level reads the
// next level's size).  Nodes are numbered in level order, the root first.
template <int DIM>
static cudaError_t build_wide(BvhBuffers& b, cudaStream_t s) {
    const int n_int = b.n_internal;
    cudaError_t e = cudaSuccess;
    std::vector<int*> lv_code, lv_src;      // per level: final codes and sources of its nodes
    std::vector<int> lv_m;
    int* roots = nullptr;
    int* next = nullptr;
    int* fr_code = nullptr;
    int* fr_src = nullptr;
    int* n_inner = nullptr;
    int* offset = nullptr;
    int m = 1, base = 0, depth = 0;
    auto cleanup = [&]() {
        for (int* p : lv_code) cudaFree(p);
        for (int* p : lv_src) cudaFree(p);
        cudaFree(roots); cudaFree(next); cudaFree(fr_code); cudaFree(fr_src); cudaFree(n_inner); cudaFree(offset);
    };
#define DW_W(x) do { e = (x); if (e != cudaSuccess) { cleanup(); return e; } } while (0)
    DW_W(cudaMalloc(&roots, sizeof(int)));
    DW_W(cudaMemsetAsync(roots, 0, sizeof(int), s));          // the binary root is node 0
    while (m > 0) {
        if (++depth > 64) { cleanup(); return cudaErrorInvalidValue; }   // a 64-level wide tree cannot happen
        int *lc = nullptr, *ls = nullptr;
        DW_W(cudaMalloc(&lc, sizeof(int) * kWide * (size_t)m));
        lv_code.push_back(lc);
        DW_W(cudaMalloc(&ls, sizeof(int) * kWide * (size_t)m));
        lv_src.push_back(ls);
        lv_m.push_back(m);
        cudaFree(fr_code); cudaFree(fr_src); cudaFree(n_inner); cudaFree(offset);
        fr_code = fr_src = n_inner = offset = nullptr;
        DW_W(cudaMalloc(&fr_code, sizeof(int) * kWide * (size_t)m));
        DW_W(cudaMalloc(&fr_src, sizeof(int) * kWide * (size_t)m));
        DW_W(cudaMalloc(&n_inner, sizeof(int) * ((size_t)m + 1)));
        DW_W(cudaMalloc(&offset, sizeof(int) * ((size_t)m + 1)));
        wide_level_kernel<<<nblk(m, 128), 128, 0, s>>>(b.node_child, b.node_count, b.node_count + n_int,
                                                       b.leaf_parent, roots, m, fr_code, fr_src, n_inner);
        DW_W(cudaMemsetAsync(n_inner + m, 0, sizeof(int), s));
        size_t tmp = 0;
        DW_W(cub::DeviceScan::ExclusiveSum(nullptr, tmp, n_inner, offset, m + 1, s));
        void* tmp_buf = nullptr;
        DW_W(cudaMalloc(&tmp_buf, tmp));
        e = cub::DeviceScan::ExclusiveSum(tmp_buf, tmp, n_inner, offset, m + 1, s);
        int next_m = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&next_m, offset + m, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(tmp_buf);
        if (e != cudaSuccess) { cleanup(); return e; }
        cudaFree(next);
        next = nullptr;
        if (next_m > 0) DW_W(cudaMalloc(&next, sizeof(int) * (size_t)next_m));
        wide_assign_kernel<<<nblk(m, 128), 128, 0, s>>>(fr_code, fr_src, offset, m, base + m, lc, ls, next);
        DW_W(cudaGetLastError());
        base += m;
        m = next_m;
        std::swap(roots, next);
    }
    const int n_wide = base;
    if (n_wide > b.wide_cap) {
        cudaFree(b.wnodes); cudaFree(b.wsrc);
        b.wnodes = nullptr; b.wsrc = nullptr; b.wide_cap = 0;
        DW_W(cudaMalloc(&b.wnodes, sizeof(float) * WideLayout<3>::kFloats * (size_t)n_wide));
        DW_W(cudaMalloc(&b.wsrc, sizeof(int) * 2 * kWide * (size_t)n_wide));   // sources, then codes
        b.wide_cap = n_wide;
    }
    b.n_wide = n_wide;
    b.wide_depth = depth;
    b.wide_ok = 31 * b.wide_depth + 1 <= kWideStack;
    int* wcode = b.wsrc + kWide * (size_t)n_wide;
    size_t at = 0;
    for (size_t l = 0; l < lv_m.size(); ++l) {
        const size_t n = kWide * (size_t)lv_m[l];
        DW_W(cudaMemcpyAsync(b.wsrc + at, lv_src[l], sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
        DW_W(cudaMemcpyAsync(wcode + at, lv_code[l], sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
        at += n;
    }
    wide_refit_kernel<DIM><<<nblk((long long)n_wide * kWide, 256), 256, 0, s>>>(b.nodes, b.prims, b.wsrc, wcode,
                                                                               n_wide, b.wnodes);
    DW_W(cudaGetLastError());
    DW_W(cudaStreamSynchronize(s));      // the level buffers are freed next
    cleanup();
#undef DW_W
    return cudaSuccess;
}

template <int DIM>
static cudaError_t build_impl(BvhBuffers& b, const float* vert, const int* elem, int n, cudaStream_t s) {
    b.n_elem = n;
    float* stats = b.stats;
    int* count = reinterpret_cast<int*>(b.stats + 2);
    cudaError_t e = cudaMemsetAsync(b.stats, 0, sizeof(float) * 2 + sizeof(int) * 4, s);
    if (e != cudaSuccess) return e;
    const int gb = min(nblk(n, 256), 1024);
    size_kernel<DIM><<<gb, 256, 0, s>>>(vert, elem, n, stats);
    count_big_kernel<DIM><<<gb, 256, 0, s>>>(vert, elem, n, stats, count);
    int host[3] = {0, 0, 0};
    e = cudaMemcpyAsync(host, count, sizeof(int) * 3, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    int n_big = host[0];
    const int split = (n_big > 0 && n_big <= kMaxBig && n_big < n) ? 1 : 0;
    if (!split) n_big = 0;
    float r_small, r_all;
    memcpy(&r_small, &host[1], sizeof(float));
    memcpy(&r_all, &host[2], sizeof(float));
    // margin for the FP32 rounding of the Morton quantisation
    b.r_max = (split ? r_small : r_all) * 1.0001f + 1e-6f;
    const int nt = n - n_big;
    b.n_big = n_big;
    b.n_tree = nt;
    e = cudaMemsetAsync(b.bounds, 0xff, sizeof(unsigned int) * DIM, s);   // min slots
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b.bounds + DIM, 0, sizeof(unsigned int) * DIM, s);             // max slots
    if (e != cudaSuccess) return e;
    bounds_kernel<DIM><<<gb, 256, 0, s>>>(vert, elem, n, stats, split, b.bounds);
    morton_kernel<DIM><<<nblk(n, 256), 256, 0, s>>>(vert, elem, n, b.bounds, stats, split, b.keys, b.vals);
    size_t tmp = b.sort_tmp_bytes;
    e = cub::DeviceRadixSort::SortPairs(b.sort_tmp, tmp, b.keys, b.keys_sorted, b.vals, b.vals_sorted, n, 0, 32, s);
    if (e != cudaSuccess) return e;
    if (nt >= 2) {
        b.n_internal = nt - 1;
        radix_tree_kernel<DIM><<<nblk(nt - 1, 256), 256, 0, s>>>(b.keys_sorted, nt, b.node_child, b.node_parent,
                                                                 b.leaf_parent, b.bounds, b.node_cell,
                                                                 b.node_count, b.node_count + (nt - 1));
        e = cudaMemsetAsync(b.counters, 0, sizeof(int) * (size_t)(nt - 1), s);
        if (e != cudaSuccess) return e;
        refit_kernel<DIM><<<nblk(nt, 256), 256, 0, s>>>(vert, elem, b.vals_sorted, nt, b.node_child,
                                                        b.node_parent, b.leaf_parent, b.counters, b.nodes);
        finalize_kernel<DIM><<<nblk(n, 256), 256, 0, s>>>(vert, elem, b.vals_sorted, n, b.node_child,
                                                          b.node_parent, nt - 1, b.nodes, b.prims, b.prim_elem,
                                                          b.leaf_of_elem);
        e = build_wide<DIM>(b, s);
        if (e != cudaSuccess) return e;
    } else {
        b.n_wide = 0;
        b.wide_depth = 0;
        b.wide_ok = true;     // nothing to search beyond the single leaf
        b.n_internal = nt;    // 1: a single-leaf node; 0: no tree
        if (nt == 1) single_leaf_kernel<DIM><<<1, 1, 0, s>>>(vert, elem, b.vals_sorted, b.nodes, b.leaf_parent,
                                                             b.node_cell);
        finalize_kernel<DIM><<<nblk(n, 256), 256, 0, s>>>(vert, elem, b.vals_sorted, n, nullptr, nullptr, 0,
                                                          b.nodes, b.prims, b.prim_elem, b.leaf_of_elem);
    }
    return cudaGetLastError();
}

cudaError_t bvh_build(BvhBuffers& b, int dim, const float* vert, const int* elem, int n_elem, cudaStream_t s) {
    cudaError_t e = bvh_reserve(b, dim, n_elem);
    if (e != cudaSuccess) return e;
    b.cells_ok = false;
    e = dim == 2 ? build_impl<2>(b, vert, elem, n_elem, s) : build_impl<3>(b, vert, elem, n_elem, s);
    b.cells_ok = e == cudaSuccess;
    return e;
}

template <int DIM>
static cudaError_t refit_impl(BvhBuffers& b, const float* vert, const int* elem, cudaStream_t s) {
    const int n = b.n_elem, nt = b.n_tree;
    if (n <= 0) return cudaSuccess;
    if (nt >= 2) {
        cudaError_t e = cudaMemsetAsync(b.counters, 0, sizeof(int) * (size_t)(nt - 1), s);
        if (e != cudaSuccess) return e;
        refit_kernel<DIM><<<nblk(nt, 256), 256, 0, s>>>(vert, elem, b.vals_sorted, nt, b.node_child,
                                                        b.node_parent, b.leaf_parent, b.counters, b.nodes);
        finalize_kernel<DIM><<<nblk(n, 256), 256, 0, s>>>(vert, elem, b.vals_sorted, n, b.node_child,
                                                          b.node_parent, nt - 1, b.nodes, b.prims, b.prim_elem,
                                                          b.leaf_of_elem);
        if (b.n_wide > 0)
            wide_refit_kernel<DIM><<<nblk((long long)b.n_wide * kWide, 256), 256, 0, s>>>(
                b.nodes, b.prims, b.wsrc, b.wsrc + kWide * (size_t)b.n_wide, b.n_wide, b.wnodes);
    } else {
        if (nt == 1) single_leaf_kernel<DIM><<<1, 1, 0, s>>>(vert, elem, b.vals_sorted, b.nodes, b.leaf_parent,
                                                             b.node_cell);
        finalize_kernel<DIM><<<nblk(n, 256), 256, 0, s>>>(vert, elem, b.vals_sorted, n, nullptr, nullptr, 0,
                                                          b.nodes, b.prims, b.prim_elem, b.leaf_of_elem);
    }
    b.cells_ok = false;
    return cudaGetLastError();
}

cudaError_t bvh_refit(BvhBuffers& b, const float* vert, const int* elem, cudaStream_t s) {
    return b.dim == 2 ? refit_impl<2>(b, vert, elem, s) : refit_impl<3>(b, vert, elem, s);
}

static BvhView view_of(const BvhBuffers& b) {
    BvhView v;
    v.nodes = b.nodes;
    v.prims = b.prims;
    v.root = 0;
    v.n_internal = b.n_internal;
    v.n_tree = b.n_tree;
    v.n_big = b.n_big;
    v.climb = 0;
    v.leaf_parent = b.leaf_parent;
    v.node_cell = b.node_cell;
    v.r_max = b.r_max;
    return v;
}

cudaError_t launch_closest(const BvhBuffers& b, int n, const float* p, const int* hint_elem, float* dist,
                           int* elem_out, float* bary, int* err, DevCounters* ctr, int traversal, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    BvhView v = view_of(b);
    if (traversal == 2 && b.wide_ok) {
        const WideView wv{b.wnodes, b.prims, b.n_wide, b.n_tree};
        const size_t smem = sizeof(float2) * kWideStack * (128 / 32);
        if (b.dim == 2) closest_wide_kernel<2><<<nblk(n, 128), 128, smem, s>>>(v, wv, b.prim_elem, b.leaf_of_elem, n, p, hint_elem, dist, elem_out, bary, err, ctr);
        else closest_wide_kernel<3><<<nblk(n, 128), 128, smem, s>>>(v, wv, b.prim_elem, b.leaf_of_elem, n, p, hint_elem, dist, elem_out, bary, err, ctr);
        return cudaGetLastError();
    }
    v.climb = traversal == 1 ? 1 : 0;
    if (b.dim == 2) closest_kernel<2><<<nblk(n, 128), 128, 0, s>>>(v, b.prim_elem, b.leaf_of_elem, n, p, hint_elem, dist, elem_out, bary, err, ctr);
    else closest_kernel<3><<<nblk(n, 128), 128, 0, s>>>(v, b.prim_elem, b.leaf_of_elem, n, p, hint_elem, dist, elem_out, bary, err, ctr);
    return cudaGetLastError();
}

cudaError_t launch_inside(const BvhBuffers& b, int n, const float* p, int* inside, cudaStream_t s,
                          const float* prev, float* prev_out) {
    if (n <= 0) return cudaSuccess;
    if (b.dim == 2) inside_kernel<2><<<nblk(32LL * n, 128), 128, 0, s>>>(view_of(b), n, p, inside, prev, prev_out);
    else inside_kernel<3><<<nblk(32LL * n, 128), 128, 0, s>>>(view_of(b), n, p, inside, prev, prev_out);
    return cudaGetLastError();
}

cudaError_t launch_philox(int n, const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    philox_kernel<<<nblk(n, 256), 256, 0, s>>>(n, ctr, k0, k1, out);
    return cudaGetLastError();
}

cudaError_t launch_apply_params(const float* vert_ref, const float* jac, const float* theta, float* vert,
                                int n_rows, int n_param, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    apply_params_kernel<<<nblk(n_rows, 256), 256, 0, s>>>(vert_ref, jac, theta, vert, n_rows, n_param);
    return cudaGetLastError();
}

}  // namespace dwos
