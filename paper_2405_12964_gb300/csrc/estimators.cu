// Estimator reductions over per-walk records (FP64 sums).
//
//  reduce_u     per-point mean and standard error of u (Sec. 3.3)
//  reduce_udot  forward-mode udot per point and parameter (Sec. 4.1, the
//               N-vector of one walk rebuilt from its record and the vertex
//               Jacobians)
//  scatter      reverse mode (Sec. 4.3): a weight per walk (VJP cotangent, or
//               the U-statistic product weight of Eq. (ustatistics) in batches
//               of B) times the walk's boundary term, scattered into per-vertex
//               FP64 accumulators a_v (d values) and s_v, aggregated per block
//               in shared memory before the global atomics
//  gemv         the adjoint map grad_theta = sum_v J_v^T a_v + sum_v dg_v s_v
//  loss         1/2 sum_p (mean_p - uref_p)^2
#include "dwos_device.cuh"
#include "dwos_internal.h"

namespace dwos {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// u of walk i (of point p), with the control variate subtracted when one is given.
__device__ __forceinline__ double walk_u(const dwos_record* __restrict__ rec, long long i, int p, const CvView cv) {
    double u = rec[i].u;
    if (cv.sample) {
        const float4 s = cv.end ? cv.end[i] : cv.sample[i];
        if (s.x == s.x) {
            double dot = (double)cv.grad[p * cv.dim] * (s.x - cv.xq[p * cv.dim]) +
                         (double)cv.grad[p * cv.dim + 1] * (s.y - cv.xq[p * cv.dim + 1]);
            if (cv.dim == 3) dot += (double)cv.grad[p * 3 + 2] * (s.z - cv.xq[p * 3 + 2]);
            u -= dot;
        }
    }
    return u;
}

// The same in FP32, for the scatter's per-walk weights.
__device__ __forceinline__ float walk_u32(const dwos_record* __restrict__ rec, long long i, int p, const CvView cv) {
    float u = rec[i].u;
    if (cv.sample) {
        const float4 s = cv.end ? cv.end[i] : cv.sample[i];
        if (s.x == s.x) {
            float dot = cv.grad[p * cv.dim] * (s.x - cv.xq[p * cv.dim]) +
                        cv.grad[p * cv.dim + 1] * (s.y - cv.xq[p * cv.dim + 1]);
            if (cv.dim == 3) dot += cv.grad[p * 3 + 2] * (s.z - cv.xq[p * 3 + 2]);
            u -= dot;
        }
    }
    return u;
}

// Mean (and standard error) of the first `used` walks of each point's W.
__global__ void reduce_u_kernel(const dwos_record* __restrict__ rec, int W, int used, double* mean, double* se,
                                CvView cv) {
    const int p = blockIdx.x;
    double s = 0.0, s2 = 0.0;
    for (int w = threadIdx.x; w < used; w += blockDim.x) {
        const double u = walk_u(rec, (long long)p * W + w, p, cv);
        s += u;
        s2 += u * u;
    }
    __shared__ double sh[2][32];
    s = warp_sum(s);
    s2 = warp_sum(s2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][warp] = s; sh[1][warp] = s2; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        s = lane < nw ? sh[0][lane] : 0.0;
        s2 = lane < nw ? sh[1][lane] : 0.0;
        s = warp_sum(s);
        s2 = warp_sum(s2);
        if (lane == 0) {
            const double m = s / used;
            mean[p] = m;
            if (se) {
                const double var = used > 1 ? fmax(s2 - used * m * m, 0.0) / (used - 1) : 0.0;
                se[p] = sqrt(var / used);
            }
        }
    }
}

// Forward-mode derivative of one walk for parameter j.
template <int DIM>
__device__ __forceinline__ double walk_udot(const dwos_record& r, const int* __restrict__ elem,
                                            const float* __restrict__ jac, const float* __restrict__ dg, int N,
                                            int j) {
    if (r.elem < 0) return 0.0;
    const float w[3] = {1.0f - r.b1 - r.b2, r.b1, r.b2};
    double v = 0.0;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        const int vid = __ldg(elem + DIM * r.elem + i);
        const float* J = jac + (size_t)vid * DIM * N + j;
        float cj = 0.0f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) cj = fmaf(r.c[k], __ldg(J + (size_t)k * N), cj);
        if (dg) cj += __ldg(dg + (size_t)vid * N + j);
        v += (double)w[i] * cj;
    }
    return v;
}

template <int DIM>
__global__ void reduce_udot_kernel(const dwos_record* __restrict__ rec, const int* __restrict__ elem,
                                   const float* __restrict__ jac, const float* __restrict__ dg, int N, int W,
                                   double* mean, double* se) {
    const int p = blockIdx.x;
    const int j = blockIdx.y * 32 + threadIdx.x;
    double s = 0.0, s2 = 0.0;
    if (j < N) {
        for (int w = threadIdx.y; w < W; w += blockDim.y) {
            const dwos_record r = rec[(size_t)p * W + w];
            const double v = walk_udot<DIM>(r, elem, jac, dg, N, j);
            s += v;
            s2 += v * v;
        }
    }
    __shared__ double sh[2][8][33];
    sh[0][threadIdx.y][threadIdx.x] = s;
    sh[1][threadIdx.y][threadIdx.x] = s2;
    __syncthreads();
    if (threadIdx.y == 0 && j < N) {
        for (int y = 1; y < blockDim.y; ++y) { s += sh[0][y][threadIdx.x]; s2 += sh[1][y][threadIdx.x]; }
        const double m = s / W;
        mean[(size_t)p * N + j] = m;
        if (se) {
            const double var = W > 1 ? fmax(s2 - W * m * m, 0.0) / (W - 1) : 0.0;
            se[(size_t)p * N + j] = sqrt(var / W);
        }
    }
}

// Reverse-mode scatter.  Each block takes a contiguous range of walks (whole
// U-statistic batches), computes every walk's weight, and accumulates the
// weighted boundary terms per vertex in a shared-memory hash table (open
// addressing, a few probes; a walk whose vertex finds no slot goes straight
// to global memory).  The table is then flushed with one FP64 atomic per
// distinct vertex and value, so vertices that many walks reach (an enclosing
// box, a coarse mesh) cost one global atomic per block instead of one per walk.
// A walk's weight and its terms, and their sum over the lanes of a warp that
// hold the same vertex, are FP32 like the walk values they come from (GB300's
// FP64 rate is a small fraction of its FP32 rate); the table and the global
// accumulators that sum them over walks are FP64.
constexpr int kSlots = 1024;

// Position of the n-th (0-based) set bit of m, or -1.
__device__ __forceinline__ int nth_set_bit(unsigned m, int n) {
    if (n >= __popc(m)) return -1;
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (n >= c) { n -= c; m >>= w; pos += w; }
    }
    return pos;
}

constexpr int kProbes = 8;
constexpr int kUSlots = 64;   // per-point u sums a block keeps in shared memory

// G: the data-derivative sums s_v (acc_g) are wanted too (DIM + 1 values per vertex, else DIM).
template <int DIM, bool G>
__global__ void __launch_bounds__(256) scatter_kernel(const dwos_record* __restrict__ rec,
                                                      const int* __restrict__ elem, int n_points, int W, int B,
                                                      int mode, const float* __restrict__ cot_or_uref,
                                                      const double* __restrict__ umean,
                                                      const float* __restrict__ pweight,
                                                      const unsigned char* __restrict__ active,
                                                      long long walks_per_block, double* __restrict__ acc_vert,
                                                      double* __restrict__ acc_g, CvView cv,
                                                      double* __restrict__ usum, double* __restrict__ zero_out,
                                                      int n_zero) {
    constexpr int NV = G ? DIM + 1 : DIM;
    if (zero_out && blockIdx.x == 0)      // an output the next kernel accumulates into
        for (int i = threadIdx.x; i < n_zero; i += blockDim.x) zero_out[i] = 0.0;
    __shared__ int keys[kSlots];
    __shared__ double vals[kSlots][NV];
    __shared__ double usl[kUSlots];
    const long long total = (long long)n_points * W;
    const long long begin = (long long)blockIdx.x * walks_per_block;
    const long long end = min(begin + walks_per_block, total);
    // the block's walks cover points p_first .. p_first + n_pb - 1
    const int p_first = (int)(begin / W);
    const int n_pb = end > begin ? (int)((end - 1) / W) - p_first + 1 : 0;
    const bool uslots = usum && n_pb <= kUSlots;
    for (int i = threadIdx.x; i < kSlots; i += blockDim.x) {
        keys[i] = -1;
#pragma unroll
        for (int k = 0; k < NV; ++k) vals[i][k] = 0.0;
    }
    for (int i = threadIdx.x; i < kUSlots; i += blockDim.x) usl[i] = 0.0;
    __syncthreads();
    for (long long base = begin; base < end; base += blockDim.x) {
        const long long i = base + threadIdx.x;
        const bool valid = i < end;
        dwos_record r;
        if (valid) r = rec[i];
        else { r.u = 0.0f; r.elem = -1; r.b1 = 0.0f; r.b2 = 0.0f; r.c[0] = r.c[1] = r.c[2] = 0.0f; r.meta = 0; }
        const int p = valid ? (int)(i / W) : 0;
        const float u = valid ? walk_u32(rec, i, p, cv) : 0.0f;
        float wt;
        if (mode == 0) {
            wt = valid ? cot_or_uref[p] / (float)W : 0.0f;
        } else if (mode == 2) {
            // correlated product, Eq. (correlated_product): (mean u - uref) mean udot, all W walks
            wt = valid ? (float)(umean[p] - (double)cot_or_uref[p]) / (float)W : 0.0f;
        } else if (mode == 3) {
            // uncorrelated product, Eq. (uncorrelated_product): u from the first W/2 walks,
            // udot from the other W/2
            const int M = W / 2;
            wt = (valid && (int)(i % W) >= M) ? (float)(umean[p] - (double)cot_or_uref[p]) / (float)M : 0.0f;
        } else {
            // U-statistic weight, Eq. (ustatistics): u*udot is estimated by
            // sum_m udot_m (S - u_m)/(B(B-1)), uref*udot by uref sum_m udot_m / B;
            // each batch is one of W/B estimates of the point's derivative.
            float S = u;
            for (int o = B >> 1; o > 0; o >>= 1) S += __shfl_xor_sync(kFull, S, o);
            const float ur = valid ? cot_or_uref[p] : 0.0f;
            wt = ((S - u) / (float)(B * (B - 1)) - ur / (float)B) / (float)(W / B);
        }
        if (pweight && valid) wt *= pweight[p];     // quadrature weight of the point
        const bool hit = valid && r.elem >= 0;
        const float wv[3] = {1.0f - r.b1 - r.b2, r.b1, r.b2};
        const int lane = threadIdx.x & 31;
        if (usum) {   // per-point sum of u: the warp's walks of one point summed in FP32, then in FP64
            const int p0 = __shfl_sync(kFull, p, 0);
            if (__all_sync(kFull, !valid || p == p0)) {
                float su = u;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) su += __shfl_xor_sync(kFull, su, o);
                if (lane == 0 && valid) atomicAdd(uslots ? usl + (p0 - p_first) : usum + p0, (double)su);
            } else if (valid) {
                atomicAdd(uslots ? usl + (p - p_first) : usum + p, (double)u);
            }
        }
#pragma unroll
        for (int sidx = 0; sidx < DIM; ++sidx) {
            int vid = hit ? __ldg(elem + DIM * r.elem + sidx) : -1;
            if (active && vid >= 0 && !__ldg(active + vid)) vid = -1;   // cannot reach the gradient
            if (!__any_sync(kFull, vid >= 0)) continue;
            const float ws = vid >= 0 ? wt * wv[sidx] : 0.0f;
            float val[NV];
#pragma unroll
            for (int k = 0; k < DIM; ++k) val[k] = ws * r.c[k];
            if (G) val[NV - 1] = ws;
            // sum over the lanes that hold the same vertex: a log-step tree over
            // each peer group (lane of rank j adds the partial sum of rank j + off)
            const unsigned peers = __match_any_sync(kFull, vid);
            if (__any_sync(kFull, vid >= 0 && __popc(peers) > 1)) {
                const int rank = __popc(peers & ((1u << lane) - 1u));
                for (int off = 1; off < 32; off <<= 1) {
                    const int src = nth_set_bit(peers, rank + off);
                    const bool has = src >= 0;
#pragma unroll
                    for (int k = 0; k < NV; ++k) {
                        const float t = __shfl_sync(kFull, val[k], has ? src : lane);
                        if (has) val[k] += t;
                    }
                }
            }
            if (vid < 0 || lane != __ffs(peers) - 1) continue;
            unsigned h = ((unsigned)vid * 2654435761u) >> 22;   // 10-bit hash
            bool done = false;
            for (int probe = 0; probe < kProbes && !done; ++probe) {
                const int slot = (int)((h + probe) & (kSlots - 1));
                const int prev = atomicCAS(&keys[slot], -1, vid);
                if (prev == -1 || prev == vid) {
#pragma unroll
                    for (int k = 0; k < NV; ++k) atomicAdd(&vals[slot][k], (double)val[k]);
                    done = true;
                }
            }
            if (!done) {
#pragma unroll
                for (int k = 0; k < DIM; ++k) atomicAdd(acc_vert + (size_t)vid * DIM + k, (double)val[k]);
                if (G) atomicAdd(acc_g + vid, (double)val[NV - 1]);
            }
        }
    }
    __syncthreads();
    if (uslots)
        for (int i = threadIdx.x; i < n_pb; i += blockDim.x) atomicAdd(usum + p_first + i, usl[i]);
    for (int i = threadIdx.x; i < kSlots; i += blockDim.x) {
        const int vid = keys[i];
        if (vid < 0) continue;
#pragma unroll
        for (int k = 0; k < DIM; ++k) atomicAdd(acc_vert + (size_t)vid * DIM + k, vals[i][k]);
        if (G) atomicAdd(acc_g + vid, vals[i][NV - 1]);
    }
}

__global__ void vertex_active_kernel(const float* __restrict__ jac, const float* __restrict__ dg, int n_vert,
                                     int dim, int n_param, unsigned char* __restrict__ out) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_vert) return;
    bool any = false;
    if (jac) {
        const float* row = jac + (size_t)v * dim * n_param;
        for (int i = 0; i < dim * n_param && !any; ++i) any = row[i] != 0.0f;
    }
    if (dg) {
        const float* row = dg + (size_t)v * n_param;
        for (int i = 0; i < n_param && !any; ++i) any = row[i] != 0.0f;
    }
    out[v] = any ? 1 : 0;
}

// grad[j] += sum over rows r (= vertex*dim + k) of J[r][j] a[r], plus sum_v dg[v][j] s[v].
__global__ void gemv_kernel(const float* __restrict__ jac, const float* __restrict__ dg,
                            const double* __restrict__ acc_vert, const double* __restrict__ acc_g, int n_vert,
                            int dim, int N, double* __restrict__ grad) {
    const int j = blockIdx.y * 32 + threadIdx.x;
    const long long rows = (long long)n_vert * dim;
    double s = 0.0;
    if (j < N) {
        for (long long r = (long long)blockIdx.x * blockDim.y + threadIdx.y; r < rows;
             r += (long long)gridDim.x * blockDim.y) {
            const double a = acc_vert[r];
            if (a != 0.0) s += (double)__ldg(jac + r * N + j) * a;
        }
        if (dg && acc_g) {
            for (long long v = (long long)blockIdx.x * blockDim.y + threadIdx.y; v < n_vert;
                 v += (long long)gridDim.x * blockDim.y) {
                const double a = acc_g[v];
                if (a != 0.0) s += (double)__ldg(dg + v * N + j) * a;
            }
        }
    }
    __shared__ double sh[8][33];
    sh[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && j < N) {
        for (int y = 1; y < blockDim.y; ++y) s += sh[y][threadIdx.x];
        atomicAdd(grad + j, s);
    }
}

// mean[p] * scale is the point's mean (scale 1 / W for per-point sums); it is
// also written to mean_out when given.
__global__ void loss_kernel(const double* mean, const float* uref, const float* pweight, int n, double* loss,
                            double scale, double* mean_out) {
    double s = 0.0;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const double m = mean[p] * scale;
        if (mean_out) mean_out[p] = m;
        const double e = m - (double)uref[p];
        s += 0.5 * e * e * (pweight ? (double)pweight[p] : 1.0);
    }
    __shared__ double sh[32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        s = warp_sum(s);
        if (threadIdx.x == 0) *loss = s;
    }
}

}  // namespace

cudaError_t launch_reduce_u(const dwos_record* rec, int n_points, int W, double* mean, double* se, cudaStream_t s,
                            const CvView* cv, int used) {
    if (n_points <= 0) return cudaSuccess;
    const CvView none{nullptr, nullptr, nullptr, 2, nullptr};
    reduce_u_kernel<<<n_points, 256, 0, s>>>(rec, W, used > 0 && used <= W ? used : W, mean, se, cv ? *cv : none);
    return cudaGetLastError();
}

__global__ void pack_samples_kernel(const dwos_record* __restrict__ rec, float4* __restrict__ samples, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 s = samples[i];
    if (s.x == s.x) s.w = rec[i].u - s.w;
    samples[i] = s;
}

// Training rows of the control-variate network from one gradient step's walks,
// thinned to the walks off, off + stride, ...  Row r < n_rows (walk i = off + r
// stride) trains the u head on (x1, estimate of u at x1) where the main walk
// moved; row n_rows + r trains the du/dn head at the walk's hit point xbar on
// y = r_i / disp_n with r_i = u_plain - g(xbar) - disp_t and g(xbar) = u_off +
// h du/dn, the least-squares fit of the nested walks' normal displacement
// (weight |disp_n|, scaled afterwards).  Accumulates sum r_i^2 and the hit
// count for that scale.
__global__ void cv_rows_kernel(const float4* __restrict__ samples, const dwos_walk_debug* __restrict__ dbg,
                               long long n_rows, long long off, long long stride, float h, float* __restrict__ x,
                               float* __restrict__ t, float* __restrict__ m, double* __restrict__ acc) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double r2 = 0.0, cnt = 0.0;
    if (r < n_rows) {
        const long long i = off + r * stride;
        const float4 s = samples[i];
        const bool ok = s.x == s.x;
        x[2 * r] = ok ? s.x : 0.0f;
        x[2 * r + 1] = ok ? s.y : 0.0f;
        t[2 * r] = ok ? s.w : 0.0f;
        t[2 * r + 1] = 0.0f;
        m[2 * r] = ok ? 1.0f : 0.0f;
        m[2 * r + 1] = 0.0f;
        if (dbg) {
            const dwos_walk_debug d = dbg[i];
            const bool hit = (d.n[0] != 0.0f || d.n[1] != 0.0f) && fabsf(d.disp_n) > 1e-7f;
            const float g = d.u_off + h * d.dudn;
            const float res = hit ? d.u_plain - g - d.disp_t : 0.0f;
            const long long q = n_rows + r;
            x[2 * q] = hit ? d.xbar[0] : 0.0f;
            x[2 * q + 1] = hit ? d.xbar[1] : 0.0f;
            t[2 * q] = 0.0f;
            t[2 * q + 1] = hit ? res / d.disp_n : 0.0f;
            m[2 * q] = 0.0f;
            m[2 * q + 1] = hit ? fabsf(d.disp_n) : 0.0f;     // times the scale below
            r2 = (double)res * res;
            cnt = hit ? 1.0 : 0.0;
        }
    }
    if (!dbg) return;
    for (int o = 16; o > 0; o >>= 1) {
        r2 += __shfl_xor_sync(0xffffffffu, r2, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0 && cnt > 0.0) {
        atomicAdd(acc, r2);
        atomicAdd(acc + 1, cnt);
    }
}

// du/dn rows' weights times sqrt(q_weight / mean r^2): the two heads' losses on
// a common scale whatever the size of the nested residuals.
__global__ void cv_scale_kernel(long long n_rows, float q_weight, const double* __restrict__ acc,
                                float* __restrict__ m) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    const double mean_r2 = acc[0] / fmax(acc[1], 1.0);
    const float scale = (float)sqrt((double)q_weight / fmax(mean_r2, 1e-12));
    m[2 * (n_rows + r) + 1] *= scale;
}

cudaError_t launch_cv_rows(const float4* samples, const dwos_walk_debug* dbg, long long n_rows, long long off,
                           long long stride, float h, float q_weight, float* x, float* t, float* m, double* acc,
                           cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    if (dbg) {
        cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), s);
        if (e != cudaSuccess) return e;
    }
    const unsigned blocks = (unsigned)((n_rows + 255) / 256);
    cv_rows_kernel<<<blocks, 256, 0, s>>>(samples, dbg, n_rows, off, stride, h, x, t, m, acc);
    if (dbg) cv_scale_kernel<<<blocks, 256, 0, s>>>(n_rows, q_weight, acc, m);
    return cudaGetLastError();
}

cudaError_t launch_pack_samples(const dwos_record* rec, float4* samples, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    pack_samples_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rec, samples, n);
    return cudaGetLastError();
}

cudaError_t launch_reduce_udot(const dwos_record* rec, const int* elem, const float* jac, const float* dg, int dim,
                               int N, int n_points, int W, double* mean, double* se, cudaStream_t s) {
    if (n_points <= 0 || N <= 0) return cudaSuccess;
    dim3 grid(n_points, (N + 31) / 32), block(32, 8);
    if (dim == 2) reduce_udot_kernel<2><<<grid, block, 0, s>>>(rec, elem, jac, dg, N, W, mean, se);
    else reduce_udot_kernel<3><<<grid, block, 0, s>>>(rec, elem, jac, dg, N, W, mean, se);
    return cudaGetLastError();
}

cudaError_t launch_vertex_active(const float* jac, const float* dg, int n_vert, int dim, int n_param,
                                 unsigned char* out, cudaStream_t s) {
    if (n_vert <= 0) return cudaSuccess;
    vertex_active_kernel<<<(n_vert + 255) / 256, 256, 0, s>>>(n_param > 0 ? jac : nullptr, n_param > 0 ? dg : nullptr,
                                                              n_vert, dim, n_param, out);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const dwos_record* rec, const int* elem, int dim, int n_points, int W, int B, int mode,
                           const float* cot_or_uref, double* acc_vert, double* acc_g, cudaStream_t s,
                           const CvView* cv, const double* umean, const float* pweight,
                           const unsigned char* active, double* usum, double* zero_out, int n_zero) {
    const CvView none{nullptr, nullptr, nullptr, dim, nullptr};
    const CvView c = cv ? *cv : none;
    const long long total = (long long)n_points * W;
    if (total <= 0)
        return zero_out && n_zero > 0 ? cudaMemsetAsync(zero_out, 0, sizeof(double) * n_zero, s) : cudaSuccess;
    const int bs = 256;
    // about four blocks per SM; each block a multiple of 256 walks (whole batches)
    long long per = (total + 4 * 152 - 1) / (4 * 152);
    per = ((per + bs - 1) / bs) * bs;
    if (per < bs) per = bs;
    const long long blocks = (total + per - 1) / per;
    auto go = [&](auto kernel) {
        kernel<<<(unsigned)blocks, bs, 0, s>>>(rec, elem, n_points, W, B, mode, cot_or_uref, umean, pweight, active,
                                              per, acc_vert, acc_g, c, usum, zero_out, n_zero);
    };
    if (dim == 2) { if (acc_g) go(scatter_kernel<2, true>); else go(scatter_kernel<2, false>); }
    else { if (acc_g) go(scatter_kernel<3, true>); else go(scatter_kernel<3, false>); }
    return cudaGetLastError();
}

cudaError_t launch_gemv(const float* jac, const float* dg, const double* acc_vert, const double* acc_g, int n_vert,
                        int dim, int N, double* grad, cudaStream_t s) {
    if (N <= 0 || n_vert <= 0) return cudaSuccess;
    const int ny = (N + 31) / 32;
    const long long rows = (long long)n_vert * dim;
    long long bx = (rows + 7) / 8;
    const long long cap = 152LL * 8 / ny + 1;
    if (bx > cap) bx = cap;
    gemv_kernel<<<dim3((unsigned)bx, ny), dim3(32, 8), 0, s>>>(jac, dg, acc_vert, acc_g, n_vert, dim, N, grad);
    return cudaGetLastError();
}

cudaError_t launch_loss(const double* mean, const float* uref, int n_points, double* loss, cudaStream_t s,
                        const float* pweight, double scale, double* mean_out) {
    loss_kernel<<<1, 256, 0, s>>>(mean, uref, pweight, n_points, loss, scale, mean_out);
    return cudaGetLastError();
}

}  // namespace dwos
