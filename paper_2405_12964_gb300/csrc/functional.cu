// The volume-integrated shape functional of Eq. (functional),
//     J(theta) = int_Omega M(x) l(u(x)) dx,  l(u) = 1/2 (u - uref)^2,
// and its derivative, Eq. (functional_deriv):
//     dJ/dtheta = int_Omega M l'(u) udot dx + int_Gamma M V_n l(u) dA.
// The domain term is a Monte Carlo integral over points sampled uniformly in a
// box-shaped mask and kept if they lie in Omega (each carries the weight
// |box| / candidates, which makes the estimate unbiased); its product l'(u)
// udot comes from the U-statistic estimator with per-point weights.  On the
// boundary u = g, so the boundary term needs no walks: it is integrated per
// element with a Gauss rule that is exact for its polynomial integrand.
#include <cub/device/device_select.cuh>

#include <cmath>
#include <cstring>
#include <string>

#include "ctx.h"
#include "dwos_device.cuh"

using namespace dwos;

namespace {

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

struct Box { float lo[3], hi[3]; };

// Candidate i: Philox4x32-10 with key = seed, counter = (i, 0, 0, 0xD0A1),
// words 0..dim-1 mapped to (0, 1) and scaled into the box.
__global__ void candidates_kernel(int n, int dim, Box box, uint32_t k0, uint32_t k1, float* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const U4 r = philox(U4{(uint32_t)i, 0u, 0u, 0xD0A1u}, k0, k1);
    const uint32_t w[3] = {r.x, r.y, r.z};
    for (int k = 0; k < dim; ++k) out[(size_t)dim * i + k] = box.lo[k] + (box.hi[k] - box.lo[k]) * u01(w[k]);
}

__global__ void iota_kernel(int n, int* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = i;
}

__global__ void gather_points_kernel(const float* cand, const int* idx, const int* count, int dim, float* out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= *count) return;
    const int i = idx[j];
    for (int k = 0; k < dim; ++k) out[(size_t)dim * j + k] = cand[(size_t)dim * i + k];
}

// Element centres pushed back along the element's geometric normal by 1e-3 of
// the element's size; the inside test of these points orients each normal
// outward.
template <int DIM>
__global__ void offset_centres_kernel(const float* vert, const int* elem, int n_elem, float* out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_elem) return;
    float c[3] = {0, 0, 0}, n[3] = {0, 0, 0};
    const int* ev = elem + DIM * e;
    if (DIM == 2) {
        const float ax = vert[2 * ev[0]], ay = vert[2 * ev[0] + 1], bx = vert[2 * ev[1]], by = vert[2 * ev[1] + 1];
        c[0] = 0.5f * (ax + bx); c[1] = 0.5f * (ay + by);
        n[0] = by - ay; n[1] = -(bx - ax);
    } else {
        float v[3][3];
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 3; ++k) v[a][k] = vert[3 * ev[a] + k];
        for (int k = 0; k < 3; ++k) c[k] = (v[0][k] + v[1][k] + v[2][k]) / 3.0f;
        const float e1[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
        const float e2[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
        n[0] = e1[1] * e2[2] - e1[2] * e2[1]; n[1] = e1[2] * e2[0] - e1[0] * e2[2]; n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    }
    float nn = 0.0f;
    for (int k = 0; k < DIM; ++k) nn += n[k] * n[k];
    const float inv = nn > 0.0f ? rsqrtf(nn) : 0.0f;
    // |n| is the segment's length (2D) or twice the triangle's area (3D)
    const float size = DIM == 2 ? sqrtf(nn) : sqrtf(sqrtf(nn));
    const float delta = 1e-3f * size;
    for (int k = 0; k < DIM; ++k) out[DIM * e + k] = c[k] - delta * n[k] * inv;
}

// Boundary term for mapped (per-vertex) data: per element,
//     a_v += int_e M w_v l(g) n dA   (v over the element's vertices),
// so that the parameter gradient is sum_v J_v^T a_v (V_n = sum_v w_v n . J_v).
// M is the box indicator at the element's centre.  l = 1/2 (g - uref)^2 with
// both g and uref linear on the element: the integrand is cubic in the
// barycentrics; 2-point Gauss (segments) and the 6-point degree-4 rule
// (triangles) integrate it exactly.
template <int DIM>
__global__ void boundary_term_kernel(const float* vert, const int* elem, int n_elem, const float* g_vert,
                                     const float* uref_vert, const int* centre_inside, Box box, double* acc) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_elem) return;
    const int* ev = elem + DIM * e;
    float v[3][3] = {{0}};
    for (int a = 0; a < DIM; ++a)
        for (int k = 0; k < DIM; ++k) v[a][k] = vert[DIM * ev[a] + k];
    float c[3] = {0, 0, 0};
    for (int a = 0; a < DIM; ++a)
        for (int k = 0; k < DIM; ++k) c[k] += v[a][k] / DIM;
    bool in_box = true;
    for (int k = 0; k < DIM; ++k) in_box = in_box && c[k] >= box.lo[k] && c[k] <= box.hi[k];
    if (!in_box) return;
    double n[3] = {0, 0, 0}, measure;
    if (DIM == 2) {
        const double tx = (double)v[1][0] - v[0][0], ty = (double)v[1][1] - v[0][1];
        measure = sqrt(tx * tx + ty * ty);
        n[0] = ty / measure; n[1] = -tx / measure;
    } else {
        const double e1[3] = {(double)v[1][0] - v[0][0], (double)v[1][1] - v[0][1], (double)v[1][2] - v[0][2]};
        const double e2[3] = {(double)v[2][0] - v[0][0], (double)v[2][1] - v[0][1], (double)v[2][2] - v[0][2]};
        const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        measure = 0.5 * len;
        for (int k = 0; k < 3; ++k) n[k] = cr[k] / len;
    }
    if (!(measure > 0.0)) return;
    const double sgn = centre_inside[e] ? 1.0 : -1.0;   // outward: the point behind the centre is inside
    double d[3] = {0, 0, 0};                            // g - uref at the vertices
    for (int a = 0; a < DIM; ++a) d[a] = (double)g_vert[ev[a]] - (uref_vert ? (double)uref_vert[ev[a]] : 0.0);
    double wsum[3] = {0, 0, 0};                         // int_e w_a l dA
    if (DIM == 2) {
        const double t[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
        for (int q = 0; q < 2; ++q) {
            const double w[2] = {1.0 - t[q], t[q]};
            const double diff = w[0] * d[0] + w[1] * d[1];
            const double l = 0.5 * diff * diff;
            for (int a = 0; a < 2; ++a) wsum[a] += 0.5 * measure * w[a] * l;
        }
    } else {
        const double A = 0.445948490915965, WA = 0.223381589678011;
        const double B = 0.091576213509771, WB = 0.109951743655322;
        const double pts[6][3] = {{A, A, 1 - 2 * A}, {A, 1 - 2 * A, A}, {1 - 2 * A, A, A},
                                  {B, B, 1 - 2 * B}, {B, 1 - 2 * B, B}, {1 - 2 * B, B, B}};
        for (int q = 0; q < 6; ++q) {
            const double* w = pts[q];
            const double diff = w[0] * d[0] + w[1] * d[1] + w[2] * d[2];
            const double l = 0.5 * diff * diff;
            for (int a = 0; a < 3; ++a) wsum[a] += (q < 3 ? WA : WB) * measure * w[a] * l;
        }
    }
    for (int a = 0; a < DIM; ++a)
        for (int k = 0; k < DIM; ++k) atomicAdd(acc + (size_t)DIM * ev[a] + k, sgn * wsum[a] * n[k]);
}

// Boundary loss of the general shape functional (App. C), for mapped vertex data:
//     J_b = sum_e m_e int_e 1/2 (g - ub)^2 dA,
// m_e the box indicator at the element's centre.  On a Dirichlet boundary the
// du/dn terms of Eq. (general_functional_deriv) cancel (udot = gdot - V_n du/dn
// there, Eq. bvp_deriv), so its derivative is that of this sum: the element
// measure's gradient (the discrete form of the mean-curvature term) times the
// element's mean of 1/2 (g - ub)^2, plus |e| int w_a (g - ub) dg_a/dtheta.  Per
// element, exactly (g and ub linear, so the mean is a quadratic form with the
// weights (1 + delta_ab) / (n (n + 1)), n = DIM vertices):
//     acc_vert[a] += m_e Q_e d|e|/dv_a,   acc_g[a] += m_e |e| sum_b d_b (1 + delta_ab) / (n (n + 1)),
//     loss += m_e |e| Q_e,                Q_e = 1/2 sum_ab d_a d_b (1 + delta_ab) / (n (n + 1)).
template <int DIM>
__global__ void boundary_loss_kernel(const float* vert, const int* elem, int n_elem, const float* g_vert,
                                     const float* ub_vert, Box box, double* acc_vert, double* acc_g,
                                     double* loss) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    double part = 0.0;
    if (e < n_elem) {
        const int* ev = elem + DIM * e;
        double v[3][3] = {{0}};
        for (int a = 0; a < DIM; ++a)
            for (int k = 0; k < DIM; ++k) v[a][k] = vert[DIM * ev[a] + k];
        bool in_box = true;
        for (int k = 0; k < DIM; ++k) {
            float c = 0.0f;
            for (int a = 0; a < DIM; ++a) c += vert[DIM * ev[a] + k] / DIM;
            in_box = in_box && c >= box.lo[k] && c <= box.hi[k];
        }
        double meas = 0.0, dm[3][3] = {{0}};
        if (DIM == 2) {
            const double tx = v[1][0] - v[0][0], ty = v[1][1] - v[0][1];
            meas = sqrt(tx * tx + ty * ty);
            if (meas > 0.0) {
                dm[0][0] = -tx / meas; dm[0][1] = -ty / meas;
                dm[1][0] = tx / meas;  dm[1][1] = ty / meas;
            }
        } else {
            const double e1[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
            const double e2[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
            const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
            const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            meas = 0.5 * nn;
            if (nn > 0.0) {
                const double h[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
                // dA/dv_a = 1/2 nhat x (v_{a+2} - v_{a+1}), a cyclic
                for (int a = 0; a < 3; ++a) {
                    const double* p = v[(a + 1) % 3];
                    const double* q = v[(a + 2) % 3];
                    const double r[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
                    dm[a][0] = 0.5 * (h[1] * r[2] - h[2] * r[1]);
                    dm[a][1] = 0.5 * (h[2] * r[0] - h[0] * r[2]);
                    dm[a][2] = 0.5 * (h[0] * r[1] - h[1] * r[0]);
                }
            }
        }
        if (in_box && meas > 0.0) {
            double d[3] = {0, 0, 0};
            for (int a = 0; a < DIM; ++a) d[a] = (double)g_vert[ev[a]] - (ub_vert ? (double)ub_vert[ev[a]] : 0.0);
            const double wn = 1.0 / (DIM * (DIM + 1));
            double q = 0.0, wa[3] = {0, 0, 0};
            for (int a = 0; a < DIM; ++a)
                for (int b = 0; b < DIM; ++b) {
                    const double c = (a == b ? 2.0 : 1.0) * wn;
                    q += 0.5 * d[a] * d[b] * c;
                    wa[a] += d[b] * c;
                }
            part = meas * q;
            for (int a = 0; a < DIM; ++a) {
                for (int k = 0; k < DIM; ++k) atomicAdd(acc_vert + (size_t)DIM * ev[a] + k, q * dm[a][k]);
                if (acc_g) atomicAdd(acc_g + ev[a], meas * wa[a]);
            }
        }
    }
    // the loss: one FP64 atomic per warp
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(loss, part);
}

dwos_status ffail(dwos_ctx* c, dwos_status s, const std::string& m) {
    c->err = m;
    return s;
}

#define FK(call, where)                                                                            \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            cudaGetLastError();                                                                    \
            return ffail(ctx, e_ == cudaErrorMemoryAllocation ? DWOS_ERR_OOM : DWOS_ERR_CUDA,       \
                         std::string(where) + ": " + cudaGetErrorString(e_));                      \
        }                                                                                          \
    } while (0)

bool box_ok(const dwos_ctx* ctx, const float* lo, const float* hi) {
    if (!lo || !hi) return false;
    for (int k = 0; k < ctx->dim; ++k)
        if (!(std::isfinite(lo[k]) && std::isfinite(hi[k]) && hi[k] > lo[k])) return false;
    return true;
}

}  // namespace

extern "C" {

dwos_status dwos_sample_domain(dwos_ctx* ctx, int n_try, const float* box_lo, const float* box_hi, uint64_t seed,
                               float* points, int* n_inside, float* weight) {
    if (!ctx) return DWOS_ERR_INVALID_ARG;
    if (!ctx->have_boundary) return ffail(ctx, DWOS_ERR_STATE, "no boundary: call dwos_set_boundary first");
    if (ctx->n_neumann > 0) return ffail(ctx, DWOS_ERR_NOT_IMPLEMENTED, "shape functionals with a Neumann part");
    if (n_try < 1 || !points || !n_inside || !weight || !box_ok(ctx, box_lo, box_hi))
        return ffail(ctx, DWOS_ERR_INVALID_ARG, "bad arguments (box: hi > lo, finite; n_try >= 1)");
    FK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int dim = ctx->dim;
    Box box{};
    double vol = 1.0;
    for (int k = 0; k < dim; ++k) { box.lo[k] = box_lo[k]; box.hi[k] = box_hi[k]; vol *= (double)box_hi[k] - box_lo[k]; }
    float* cand = nullptr;
    int *flags = nullptr, *idx = nullptr, *count = nullptr, *seq = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    cudaStream_t s = ctx->stream;
    auto cleanup = [&]() { cudaFree(cand); cudaFree(flags); cudaFree(idx); cudaFree(count); cudaFree(tmp); cudaFree(seq); };
    cudaError_t e = cudaMalloc(&cand, sizeof(float) * dim * (size_t)n_try);
    if (e == cudaSuccess) e = cudaMalloc(&flags, sizeof(int) * (size_t)n_try);
    if (e == cudaSuccess) e = cudaMalloc(&idx, sizeof(int) * (size_t)n_try);
    if (e == cudaSuccess) e = cudaMalloc(&count, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&seq, sizeof(int) * (size_t)n_try);
    if (e == cudaSuccess) e = cub::DeviceSelect::Flagged(nullptr, tmp_bytes, seq, flags, idx, count, n_try, s);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, tmp_bytes);
    if (e == cudaSuccess) {
        candidates_kernel<<<nblk(n_try, 256), 256, 0, s>>>(n_try, dim, box, (uint32_t)seed, (uint32_t)(seed >> 32), cand);
        iota_kernel<<<nblk(n_try, 256), 256, 0, s>>>(n_try, seq);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_inside(ctx->bvh, n_try, cand, flags, s);
    if (e == cudaSuccess) e = cub::DeviceSelect::Flagged(tmp, tmp_bytes, seq, flags, idx, count, n_try, s);
    if (e == cudaSuccess) {
        gather_points_kernel<<<nblk(n_try, 256), 256, 0, s>>>(cand, idx, count, dim, points);
        e = cudaGetLastError();
    }
    int n_in = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n_in, count, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    FK(e, "domain sampling");
    ctx->launches += 4;
    *n_inside = n_in;
    *weight = (float)(vol / n_try);
    return DWOS_OK;
}

dwos_status dwos_boundary_term_l2(dwos_ctx* ctx, const float* box_lo, const float* box_hi, const float* uref_vert,
                                  double* grad_param, int mem) {
    if (!ctx) return DWOS_ERR_INVALID_ARG;
    if (!ctx->have_boundary) return ffail(ctx, DWOS_ERR_STATE, "no boundary: call dwos_set_boundary first");
    if (ctx->n_neumann > 0) return ffail(ctx, DWOS_ERR_NOT_IMPLEMENTED, "shape functionals with a Neumann part");
    if (!box_ok(ctx, box_lo, box_hi) || (ctx->n_param > 0 && !grad_param) ||
        (mem != DWOS_MEM_HOST && mem != DWOS_MEM_DEVICE))
        return ffail(ctx, DWOS_ERR_INVALID_ARG, "bad arguments");
    if (ctx->data_kind != 0)
        return ffail(ctx, DWOS_ERR_NOT_IMPLEMENTED, "the boundary term is implemented for mapped (per-vertex) data");
    FK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int dim = ctx->dim, ne = ctx->n_elem, nv = ctx->n_vert, N = ctx->n_param;
    cudaStream_t s = ctx->stream;
    Box box{};
    for (int k = 0; k < dim; ++k) { box.lo[k] = box_lo[k]; box.hi[k] = box_hi[k]; }
    float* off = nullptr;
    int* inside = nullptr;
    float* uref = nullptr;
    double* acc = nullptr;
    double* grad = nullptr;
    auto cleanup = [&]() { cudaFree(off); cudaFree(inside); cudaFree(uref); cudaFree(acc); cudaFree(grad); };
    cudaError_t e = cudaMalloc(&off, sizeof(float) * dim * (size_t)ne);
    if (e == cudaSuccess) e = cudaMalloc(&inside, sizeof(int) * (size_t)ne);
    if (e == cudaSuccess) e = cudaMalloc(&acc, sizeof(double) * dim * (size_t)nv);
    if (e == cudaSuccess) e = cudaMalloc(&grad, sizeof(double) * (size_t)(N > 0 ? N : 1));
    if (e == cudaSuccess && uref_vert) {
        e = cudaMalloc(&uref, sizeof(float) * (size_t)nv);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(uref, uref_vert, sizeof(float) * nv,
                                mem == DWOS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, sizeof(double) * dim * (size_t)nv, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(grad, 0, sizeof(double) * (size_t)(N > 0 ? N : 1), s);
    if (e == cudaSuccess) {
        if (dim == 2) offset_centres_kernel<2><<<nblk(ne, 256), 256, 0, s>>>(ctx->vert, ctx->elem, ne, off);
        else offset_centres_kernel<3><<<nblk(ne, 256), 256, 0, s>>>(ctx->vert, ctx->elem, ne, off);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_inside(ctx->bvh, ne, off, inside, s);
    if (e == cudaSuccess) {
        if (dim == 2)
            boundary_term_kernel<2><<<nblk(ne, 256), 256, 0, s>>>(ctx->vert, ctx->elem, ne, ctx->g_vert, uref, inside, box, acc);
        else
            boundary_term_kernel<3><<<nblk(ne, 256), 256, 0, s>>>(ctx->vert, ctx->elem, ne, ctx->g_vert, uref, inside, box, acc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && N > 0) e = launch_gemv(ctx->jac, nullptr, acc, nullptr, nv, dim, N, grad, s);
    if (e == cudaSuccess && N > 0)
        e = cudaMemcpyAsync(grad_param, grad, sizeof(double) * N,
                            mem == DWOS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    FK(e, "boundary term");
    ctx->launches += 4;
    return DWOS_OK;
}

dwos_status dwos_boundary_loss_l2(dwos_ctx* ctx, const float* box_lo, const float* box_hi, const float* ub_vert,
                                  double* loss, double* grad_param, int mem) {
    if (!ctx) return DWOS_ERR_INVALID_ARG;
    if (!ctx->have_boundary) return ffail(ctx, DWOS_ERR_STATE, "no boundary: call dwos_set_boundary first");
    if (ctx->n_neumann > 0) return ffail(ctx, DWOS_ERR_NOT_IMPLEMENTED, "shape functionals with a Neumann part");
    if (!box_ok(ctx, box_lo, box_hi) || !loss || (ctx->n_param > 0 && !grad_param) ||
        (mem != DWOS_MEM_HOST && mem != DWOS_MEM_DEVICE))
        return ffail(ctx, DWOS_ERR_INVALID_ARG, "bad arguments");
    if (ctx->data_kind != 0)
        return ffail(ctx, DWOS_ERR_NOT_IMPLEMENTED, "the boundary loss is implemented for mapped (per-vertex) data");
    FK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int dim = ctx->dim, ne = ctx->n_elem, nv = ctx->n_vert, N = ctx->n_param;
    const cudaMemcpyKind out_kind = mem == DWOS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaStream_t s = ctx->stream;
    Box box{};
    for (int k = 0; k < dim; ++k) { box.lo[k] = box_lo[k]; box.hi[k] = box_hi[k]; }
    float* ub = nullptr;
    double* acc = nullptr;       // n_vert * dim position sums, then n_vert data sums, then the loss
    double* grad = nullptr;
    auto cleanup = [&]() { cudaFree(ub); cudaFree(acc); cudaFree(grad); };
    const size_t nacc = (size_t)nv * dim + nv + 1;
    cudaError_t e = cudaMalloc(&acc, sizeof(double) * nacc);
    if (e == cudaSuccess) e = cudaMalloc(&grad, sizeof(double) * (size_t)(N > 0 ? N : 1));
    if (e == cudaSuccess && ub_vert) {
        e = cudaMalloc(&ub, sizeof(float) * (size_t)nv);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ub, ub_vert, sizeof(float) * nv,
                                mem == DWOS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, sizeof(double) * nacc, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(grad, 0, sizeof(double) * (size_t)(N > 0 ? N : 1), s);
    double* acc_g = ctx->dg_vert ? acc + (size_t)nv * dim : nullptr;
    double* d_loss = acc + (size_t)nv * dim + nv;
    if (e == cudaSuccess) {
        if (dim == 2)
            boundary_loss_kernel<2><<<nblk(ne, 256), 256, 0, s>>>(ctx->vert, ctx->elem, ne, ctx->g_vert, ub, box, acc, acc_g, d_loss);
        else
            boundary_loss_kernel<3><<<nblk(ne, 256), 256, 0, s>>>(ctx->vert, ctx->elem, ne, ctx->g_vert, ub, box, acc, acc_g, d_loss);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && N > 0) e = launch_gemv(ctx->jac, ctx->dg_vert, acc, acc_g, nv, dim, N, grad, s);
    if (e == cudaSuccess && N > 0) e = cudaMemcpyAsync(grad_param, grad, sizeof(double) * N, out_kind, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, d_loss, sizeof(double), out_kind, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    FK(e, "boundary loss");
    ctx->launches += N > 0 ? 2 : 1;
    return DWOS_OK;
}

}  // extern "C"
