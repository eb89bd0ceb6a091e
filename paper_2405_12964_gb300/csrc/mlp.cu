// Control-variate network: features (x, y, sin pi x, sin pi y, sin pi (x+y))
// -> 4 x 64 tanh -> 8 linear outputs (0: u, 1: du/dn).  Training runs on the
// tensor cores (mma.sync m16n8k16, BF16 inputs, FP32 accumulation): forward
// products, the back-propagated deltas and the weight gradients.  Parameters
// are kept in FP32 (Adam) and copied to BF16 for the products.  Evaluation of
// u, its spatial gradient and the du/dn head is a scalar FP32 kernel with the
// BF16 weights (it runs on a few thousand query points).
//
// Flat parameter layout: W1 (64 x 16), b1 (64), W2 (64 x 64), b2, W3, b3,
// W4, b4, W5 (8 x 64), b5 (8); W[out][in] row-major.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "../../include/dwos.h"

namespace {

constexpr int H = 64;            // hidden width
constexpr int IN = 16;           // padded input width
constexpr int OUT = 8;           // padded output width
constexpr int NP = DWOS_MLP_NPARAM;
// offsets of W_l and b_l (l = 1..5) in the flat parameter vector
__host__ __device__ constexpr int off_w(int l) { return l == 1 ? 0 : 1088 + (l - 2) * 4160; }
__host__ __device__ constexpr int off_b(int l) { return l == 1 ? 1024 : (l == 5 ? 14080 : 1088 + (l - 2) * 4160 + 4096); }
static_assert(off_b(5) + 8 == DWOS_MLP_NPARAM, "parameter layout");
constexpr int WARPS = 4;
constexpr int TILE = 16;                 // samples per warp
constexpr int BS = WARPS * TILE;         // samples per block

// BF16 weight copies: forward operand W[out][in] and backward operand W^T[in][out_pad]
struct Bf16Weights {
    __nv_bfloat16 w1[H * IN];
    __nv_bfloat16 w2[H * H], w3[H * H], w4[H * H];
    __nv_bfloat16 w5[OUT * H];
    __nv_bfloat16 t2[H * H], t3[H * H], t4[H * H];   // t_l[in][out] = W_l[out][in]
    __nv_bfloat16 t5[H * 16];                        // W5^T padded to 16 outputs
};

struct Smem {
    Bf16Weights w;
    float act[5][BS * H];     // layer inputs: act[0] = features (IN wide, stride H), act[l] = a_l
    float delta[BS * H];      // current layer's delta
    float loss[WARPS];
};

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t ld2(const __nv_bfloat16* p) {   // two adjacent BF16
    return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ void mma(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void feats(float x, float y, float* f) {
    f[0] = x;
    f[1] = y;
    f[2] = sinpif(x);
    f[3] = sinpif(y);
    f[4] = sinpif(x + y);
}

// Masked-MSE gradient over n samples, accumulated into grad (FP32, zeroed by the
// caller) and loss (FP64 sum).
__global__ void __launch_bounds__(WARPS * 32) train_kernel(const Bf16Weights* __restrict__ gw,
                                                           const float* __restrict__ params, int n,
                                                           const float* __restrict__ x, const float* __restrict__ target,
                                                           const float* __restrict__ mask, float* __restrict__ grad,
                                                           double* __restrict__ loss) {
    extern __shared__ __align__(16) unsigned char raw[];
    Smem& S = *reinterpret_cast<Smem*>(raw);
    {
        const int words = sizeof(Bf16Weights) / 4;
        const int* src = reinterpret_cast<const int*>(gw);
        int* dst = reinterpret_cast<int*>(&S.w);
        for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int s0 = blockIdx.x * BS + warp * TILE;       // first sample of this warp
    const float inv_n = 1.0f / (float)n;

    // ---- features of rows g and g + 8
    float fr[2][5];
    bool valid[2];
    for (int h = 0; h < 2; ++h) {
        const int s = s0 + g + 8 * h;
        valid[h] = s < n;
        if (valid[h]) feats(x[2 * s], x[2 * s + 1], fr[h]);
        else for (int k = 0; k < 5; ++k) fr[h][k] = 0.0f;
    }
    __syncthreads();
    // store features (FP32) for the first layer's weight gradient
    if (t == 0) {
        for (int h = 0; h < 2; ++h) {
            float* row = S.act[0] + (warp * TILE + g + 8 * h) * H;
            for (int k = 0; k < IN; ++k) row[k] = k < 5 ? fr[h][k] : 0.0f;
        }
    }
    // A fragment of the features (K = 16): columns 2t, 2t+1 and 2t+8, 2t+9
    uint32_t a[4][4];
    {
        auto fv = [&](int h, int c) { return c < 5 ? fr[h][c] : 0.0f; };
        a[0][0] = pack2(fv(0, 2 * t), fv(0, 2 * t + 1));
        a[0][1] = pack2(fv(1, 2 * t), fv(1, 2 * t + 1));
        a[0][2] = pack2(fv(0, 2 * t + 8), fv(0, 2 * t + 9));
        a[0][3] = pack2(fv(1, 2 * t + 8), fv(1, 2 * t + 9));
    }
    const __nv_bfloat16* Wf[5] = {S.w.w1, S.w.w2, S.w.w3, S.w.w4, S.w.w5};
    float acc[8][4];
    // ---- forward: four tanh layers
    for (int l = 1; l <= 4; ++l) {
        const int kin = l == 1 ? IN : H;
        const __nv_bfloat16* W = Wf[l - 1];
        const float* b = params + off_b(l);
        for (int nt = 0; nt < 8; ++nt) {
            const float b0 = b[nt * 8 + 2 * t], b1 = b[nt * 8 + 2 * t + 1];
            acc[nt][0] = b0; acc[nt][1] = b1; acc[nt][2] = b0; acc[nt][3] = b1;
        }
        for (int kt = 0; kt < kin / 16; ++kt)
            for (int nt = 0; nt < 8; ++nt) {
                const __nv_bfloat16* wr = W + (nt * 8 + g) * kin + kt * 16 + 2 * t;
                mma(acc[nt], a[kt], ld2(wr), ld2(wr + 8));
            }
        float* A = S.act[l];
        for (int nt = 0; nt < 8; ++nt) {
            for (int i = 0; i < 4; ++i) acc[nt][i] = tanhf(acc[nt][i]);
            const int c = nt * 8 + 2 * t;
            A[(warp * TILE + g) * H + c] = acc[nt][0];
            A[(warp * TILE + g) * H + c + 1] = acc[nt][1];
            A[(warp * TILE + g + 8) * H + c] = acc[nt][2];
            A[(warp * TILE + g + 8) * H + c + 1] = acc[nt][3];
        }
        for (int kt = 0; kt < 4; ++kt) {
            a[kt][0] = pack2(acc[2 * kt][0], acc[2 * kt][1]);
            a[kt][1] = pack2(acc[2 * kt][2], acc[2 * kt][3]);
            a[kt][2] = pack2(acc[2 * kt + 1][0], acc[2 * kt + 1][1]);
            a[kt][3] = pack2(acc[2 * kt + 1][2], acc[2 * kt + 1][3]);
        }
    }
    // ---- output layer (one n-tile of 8) and the loss delta
    float o[4];
    {
        const float* b = params + off_b(5);
        o[0] = b[2 * t]; o[1] = b[2 * t + 1]; o[2] = b[2 * t]; o[3] = b[2 * t + 1];
        for (int kt = 0; kt < 4; ++kt) {
            const __nv_bfloat16* wr = S.w.w5 + g * H + kt * 16 + 2 * t;
            mma(o, a[kt], ld2(wr), ld2(wr + 8));
        }
    }
    float d5[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float lsum = 0.0f;
    if (t == 0) {
        for (int h = 0; h < 2; ++h) {
            const int s = s0 + g + 8 * h;
            if (!valid[h]) continue;
            for (int k = 0; k < 2; ++k) {
                const float m = mask[2 * s + k];
                const float e = m * (o[2 * h + k] - target[2 * s + k]);
                lsum += e * e;
                d5[2 * h + k] = 2.0f * e * inv_n;
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    if (lane == 0) atomicAdd(loss, (double)lsum * (double)inv_n);

    // delta of the output layer to shared memory: delta[s][0..7]
    __syncthreads();
    {
        float* D = S.delta;
        D[(warp * TILE + g) * H + 2 * t] = d5[0];
        D[(warp * TILE + g) * H + 2 * t + 1] = d5[1];
        D[(warp * TILE + g + 8) * H + 2 * t] = d5[2];
        D[(warp * TILE + g + 8) * H + 2 * t + 1] = d5[3];
    }
    __syncthreads();

    // Weight gradient dW[out][in] = sum_s bf16(delta[s][out]) bf16(act[s][in]) over the block's
    // samples (K = 64), plus db[out] = sum_s delta[s][out].  Rows beyond `outs` are zero.
    auto weight_grad = [&](int l, int outs, int ins) {
        const float* D = S.delta;
        const float* A = S.act[l - 1];
        const int mtiles = (outs + 15) / 16, ntiles = ins / 8;
        for (int pair = warp; pair < mtiles * ntiles; pair += WARPS) {
            const int mt = pair / ntiles, nt = pair % ntiles;
            float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int kt = 0; kt < BS / 16; ++kt) {
                const int sa = kt * 16 + 2 * t;
                const int r0 = mt * 16 + g, r1 = r0 + 8;
                auto dv = [&](int s, int r) { return r < outs ? D[s * H + r] : 0.0f; };
                uint32_t af[4] = {pack2(dv(sa, r0), dv(sa + 1, r0)), pack2(dv(sa, r1), dv(sa + 1, r1)),
                                  pack2(dv(sa + 8, r0), dv(sa + 9, r0)), pack2(dv(sa + 8, r1), dv(sa + 9, r1))};
                const int col = nt * 8 + g;
                const uint32_t b0 = pack2(A[sa * H + col], A[(sa + 1) * H + col]);
                const uint32_t b1 = pack2(A[(sa + 8) * H + col], A[(sa + 9) * H + col]);
                mma(c, af, b0, b1);
            }
            float* gW = grad + off_w(l);
            const int r0 = mt * 16 + g, c0 = nt * 8 + 2 * t;
            if (r0 < outs) { atomicAdd(gW + r0 * ins + c0, c[0]); atomicAdd(gW + r0 * ins + c0 + 1, c[1]); }
            if (r0 + 8 < outs) { atomicAdd(gW + (r0 + 8) * ins + c0, c[2]); atomicAdd(gW + (r0 + 8) * ins + c0 + 1, c[3]); }
        }
        for (int r = threadIdx.x; r < outs; r += blockDim.x) {
            float sb = 0.0f;
            for (int s = 0; s < BS; ++s) sb += D[s * H + r];
            atomicAdd(grad + off_b(l) + r, sb);
        }
    };
    weight_grad(5, OUT, H);

    // ---- backward through the hidden layers
    // delta_l = (delta_{l+1} W_{l+1}) * (1 - a_l^2); the product uses W^T[in][out] as B
    uint32_t da[4][4];
    da[0][0] = pack2(d5[0], d5[1]);
    da[0][1] = pack2(d5[2], d5[3]);
    da[0][2] = 0u;
    da[0][3] = 0u;
    int ktiles = 1;
    const __nv_bfloat16* Wt[6] = {nullptr, nullptr, S.w.t2, S.w.t3, S.w.t4, S.w.t5};
    for (int l = 4; l >= 1; --l) {
        const __nv_bfloat16* T = Wt[l + 1];
        const int kout = l == 4 ? 16 : H;       // padded width of layer l+1's outputs
        float dd[8][4];
        for (int nt = 0; nt < 8; ++nt) {
            dd[nt][0] = dd[nt][1] = dd[nt][2] = dd[nt][3] = 0.0f;
            for (int kt = 0; kt < ktiles; ++kt) {
                const __nv_bfloat16* tr = T + (nt * 8 + g) * kout + kt * 16 + 2 * t;
                mma(dd[nt], da[kt], ld2(tr), ld2(tr + 8));
            }
        }
        __syncthreads();     // the previous weight gradient has finished reading S.delta
        const float* A = S.act[l];
        float* D = S.delta;
        for (int nt = 0; nt < 8; ++nt) {
            const int c = nt * 8 + 2 * t;
            const int ra = (warp * TILE + g) * H, rb = (warp * TILE + g + 8) * H;
            dd[nt][0] *= 1.0f - A[ra + c] * A[ra + c];
            dd[nt][1] *= 1.0f - A[ra + c + 1] * A[ra + c + 1];
            dd[nt][2] *= 1.0f - A[rb + c] * A[rb + c];
            dd[nt][3] *= 1.0f - A[rb + c + 1] * A[rb + c + 1];
            D[ra + c] = dd[nt][0];
            D[ra + c + 1] = dd[nt][1];
            D[rb + c] = dd[nt][2];
            D[rb + c + 1] = dd[nt][3];
        }
        for (int kt = 0; kt < 4; ++kt) {
            da[kt][0] = pack2(dd[2 * kt][0], dd[2 * kt][1]);
            da[kt][1] = pack2(dd[2 * kt][2], dd[2 * kt][3]);
            da[kt][2] = pack2(dd[2 * kt + 1][0], dd[2 * kt + 1][1]);
            da[kt][3] = pack2(dd[2 * kt + 1][2], dd[2 * kt + 1][3]);
        }
        ktiles = 4;
        __syncthreads();
        weight_grad(l, H, l == 1 ? IN : H);
    }
}

// BF16 copies (and transposes) of the FP32 parameters.
__global__ void convert_kernel(const float* __restrict__ p, Bf16Weights* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < H * IN) w->w1[i] = __float2bfloat16_rn(p[off_w(1) + i]);
    if (i < H * H) {
        const int o = i / H, in = i % H;
        w->w2[i] = __float2bfloat16_rn(p[off_w(2) + i]);
        w->w3[i] = __float2bfloat16_rn(p[off_w(3) + i]);
        w->w4[i] = __float2bfloat16_rn(p[off_w(4) + i]);
        w->t2[in * H + o] = __float2bfloat16_rn(p[off_w(2) + i]);
        w->t3[in * H + o] = __float2bfloat16_rn(p[off_w(3) + i]);
        w->t4[in * H + o] = __float2bfloat16_rn(p[off_w(4) + i]);
    }
    if (i < OUT * H) w->w5[i] = __float2bfloat16_rn(p[off_w(5) + i]);
    if (i < H * 16) {
        const int in = i / 16, o = i % 16;
        w->t5[i] = __float2bfloat16_rn(o < OUT ? p[off_w(5) + o * H + in] : 0.0f);
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// u head, d u / d(x, y) and the du/dn head at n points (scalar FP32, BF16 weights).
__global__ void eval_kernel(const Bf16Weights* __restrict__ w, const float* __restrict__ params, int n,
                            const float* __restrict__ x, float* __restrict__ u, float* __restrict__ gu,
                            float* __restrict__ q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float f[5];
    feats(x[2 * i], x[2 * i + 1], f);
    float a[5][H];
    for (int o = 0; o < H; ++o) {
        float s = params[off_b(1) + o];
        for (int k = 0; k < 5; ++k) s = fmaf(__bfloat162float(w->w1[o * IN + k]), f[k], s);
        a[1][o] = tanhf(s);
    }
    const __nv_bfloat16* Wl[5] = {nullptr, nullptr, w->w2, w->w3, w->w4};
    for (int l = 2; l <= 4; ++l)
        for (int o = 0; o < H; ++o) {
            float s = params[off_b(l) + o];
            for (int k = 0; k < H; ++k) s = fmaf(__bfloat162float(Wl[l][o * H + k]), a[l - 1][k], s);
            a[l][o] = tanhf(s);
        }
    float out0 = params[off_b(5)], out1 = params[off_b(5) + 1];
    for (int k = 0; k < H; ++k) {
        out0 = fmaf(__bfloat162float(w->w5[k]), a[4][k], out0);
        out1 = fmaf(__bfloat162float(w->w5[H + k]), a[4][k], out1);
    }
    // d u / d a_l, back to the features
    float back[H], nb[H];
    for (int k = 0; k < H; ++k) back[k] = __bfloat162float(w->w5[k]) * (1.0f - a[4][k] * a[4][k]);
    for (int l = 4; l >= 2; --l) {
        for (int k = 0; k < H; ++k) {
            float s = 0.0f;
            for (int o = 0; o < H; ++o) s = fmaf(back[o], __bfloat162float(Wl[l][o * H + k]), s);
            nb[k] = s * (1.0f - a[l - 1][k] * a[l - 1][k]);
        }
        for (int k = 0; k < H; ++k) back[k] = nb[k];
    }
    float df[5];
    for (int k = 0; k < 5; ++k) {
        float s = 0.0f;
        for (int o = 0; o < H; ++o) s = fmaf(back[o], __bfloat162float(w->w1[o * IN + k]), s);
        df[k] = s;
    }
    const float px = x[2 * i], py = x[2 * i + 1];
    const float c0 = 3.14159265358979f * cospif(px), c1 = 3.14159265358979f * cospif(py);
    const float c01 = 3.14159265358979f * cospif(px + py);
    if (u) u[i] = out0;
    if (q) q[i] = out1;
    if (gu) {
        gu[2 * i] = df[0] + df[2] * c0 + df[4] * c01;
        gu[2 * i + 1] = df[1] + df[3] * c1 + df[4] * c01;
    }
}

}  // namespace

struct dwos_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    float* p = nullptr;          // parameters (FP32)
    float* g = nullptr;          // gradient
    float* m = nullptr;          // Adam moments
    float* v = nullptr;
    double* loss = nullptr;
    Bf16Weights* w = nullptr;
    float* scratch = nullptr;    // staging for host inputs
    size_t scratch_cap = 0;
    long long step = 0;
};

namespace {

thread_local std::string g_mlp_err;

dwos_status mfail(dwos_mlp* m, dwos_status s, const std::string& e) {
    if (m) m->err = e; else g_mlp_err = e;
    return s;
}

dwos_status mcuda(dwos_mlp* m, cudaError_t e, const char* where) {
    cudaGetLastError();
    return mfail(m, e == cudaErrorMemoryAllocation ? DWOS_ERR_OOM : DWOS_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

#define MK(call, where) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return mcuda(mlp, e_, where); } while (0)

// Stage host inputs (mem = host) into device scratch; returns device pointers.
dwos_status stage(dwos_mlp* mlp, int mem, size_t n_floats, const float* const* in, float** out, int count) {
    if (mem == DWOS_MEM_DEVICE) {
        for (int i = 0; i < count; ++i) out[i] = const_cast<float*>(in[i]);
        return DWOS_OK;
    }
    size_t need = n_floats * count;
    if (need > mlp->scratch_cap) {
        cudaFree(mlp->scratch);
        mlp->scratch = nullptr;
        mlp->scratch_cap = 0;
        MK(cudaMalloc(&mlp->scratch, need * sizeof(float)), "alloc scratch");
        mlp->scratch_cap = need;
    }
    for (int i = 0; i < count; ++i) {
        out[i] = mlp->scratch + n_floats * i;
        if (in[i]) MK(cudaMemcpyAsync(out[i], in[i], n_floats * sizeof(float), cudaMemcpyHostToDevice, mlp->stream),
                      "copy input");
        else out[i] = nullptr;
    }
    return DWOS_OK;
}

dwos_status grads(dwos_mlp* mlp, int n, const float* x, const float* t, const float* mk) {
    MK(cudaMemsetAsync(mlp->g, 0, sizeof(float) * NP, mlp->stream), "zero grad");
    MK(cudaMemsetAsync(mlp->loss, 0, sizeof(double), mlp->stream), "zero loss");
    const int blocks = (n + BS - 1) / BS;
    train_kernel<<<blocks, WARPS * 32, sizeof(Smem), mlp->stream>>>(mlp->w, mlp->p, n, x, t, mk, mlp->g, mlp->loss);
    MK(cudaGetLastError(), "train kernel");
    return DWOS_OK;
}

}  // namespace

extern "C" {

dwos_status dwos_mlp_create(dwos_mlp** out, int device) {
    if (!out) return mfail(nullptr, DWOS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    dwos_mlp* mlp = new dwos_mlp();
    mlp->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMalloc(&mlp->p, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc(&mlp->g, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc(&mlp->m, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc(&mlp->v, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc(&mlp->loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&mlp->w, sizeof(Bf16Weights));
    if (e == cudaSuccess) e = cudaMemset(mlp->p, 0, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMemset(mlp->m, 0, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMemset(mlp->v, 0, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)sizeof(Smem));
    if (e != cudaSuccess) {
        g_mlp_err = std::string("mlp setup: ") + cudaGetErrorString(e);
        cudaGetLastError();
        dwos_mlp_destroy(mlp);
        return e == cudaErrorMemoryAllocation ? DWOS_ERR_OOM : DWOS_ERR_CUDA;
    }
    *out = mlp;
    return DWOS_OK;
}

void dwos_mlp_destroy(dwos_mlp* mlp) {
    if (!mlp) return;
    cudaSetDevice(mlp->device);
    if (mlp->stream) cudaStreamSynchronize(mlp->stream);
    for (void* p : {(void*)mlp->p, (void*)mlp->g, (void*)mlp->m, (void*)mlp->v, (void*)mlp->loss, (void*)mlp->w,
                    (void*)mlp->scratch})
        if (p) cudaFree(p);
    delete mlp;
}

const char* dwos_mlp_last_error(const dwos_mlp* mlp) { return mlp ? mlp->err.c_str() : g_mlp_err.c_str(); }

dwos_status dwos_mlp_set_stream(dwos_mlp* mlp, void* stream) {
    if (!mlp) return mfail(nullptr, DWOS_ERR_INVALID_ARG, "mlp is NULL");
    mlp->stream = (cudaStream_t)stream;
    return DWOS_OK;
}

dwos_status dwos_mlp_set_params(dwos_mlp* mlp, const float* params, int mem) {
    if (!mlp || !params) return mfail(mlp, DWOS_ERR_INVALID_ARG, "NULL argument");
    MK(cudaSetDevice(mlp->device), "cudaSetDevice");
    MK(cudaMemcpyAsync(mlp->p, params, sizeof(float) * NP,
                       mem == DWOS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, mlp->stream),
       "copy params");
    MK(cudaMemsetAsync(mlp->m, 0, sizeof(float) * NP, mlp->stream), "reset moments");
    MK(cudaMemsetAsync(mlp->v, 0, sizeof(float) * NP, mlp->stream), "reset moments");
    mlp->step = 0;
    convert_kernel<<<(H * H + 255) / 256, 256, 0, mlp->stream>>>(mlp->p, mlp->w);
    MK(cudaGetLastError(), "convert");
    if (mem == DWOS_MEM_HOST) MK(cudaStreamSynchronize(mlp->stream), "synchronize");
    return DWOS_OK;
}

dwos_status dwos_mlp_get_params(dwos_mlp* mlp, float* params, int mem) {
    if (!mlp || !params) return mfail(mlp, DWOS_ERR_INVALID_ARG, "NULL argument");
    MK(cudaSetDevice(mlp->device), "cudaSetDevice");
    MK(cudaMemcpyAsync(params, mlp->p, sizeof(float) * NP,
                       mem == DWOS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, mlp->stream),
       "copy params");
    if (mem == DWOS_MEM_HOST) MK(cudaStreamSynchronize(mlp->stream), "synchronize");
    return DWOS_OK;
}

dwos_status dwos_mlp_loss_grad(dwos_mlp* mlp, int n, const float* x, const float* target, const float* mask,
                               float* grad, double* loss, int mem) {
    if (!mlp || n < 1 || !x || !target || !mask) return mfail(mlp, DWOS_ERR_INVALID_ARG, "bad arguments");
    MK(cudaSetDevice(mlp->device), "cudaSetDevice");
    const float* in[3] = {x, target, mask};
    float* d[3];
    if (dwos_status s = stage(mlp, mem, 2 * (size_t)n, in, d, 3)) return s;
    if (dwos_status s = grads(mlp, n, d[0], d[1], d[2])) return s;
    const cudaMemcpyKind k = mem == DWOS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (grad) MK(cudaMemcpyAsync(grad, mlp->g, sizeof(float) * NP, k, mlp->stream), "copy grad");
    if (loss) MK(cudaMemcpyAsync(loss, mlp->loss, sizeof(double), k, mlp->stream), "copy loss");
    if (mem == DWOS_MEM_HOST) MK(cudaStreamSynchronize(mlp->stream), "synchronize");
    return DWOS_OK;
}

dwos_status dwos_mlp_train_step(dwos_mlp* mlp, int n, const float* x, const float* target, const float* mask,
                                float lr, double* loss, int mem) {
    if (!mlp || n < 1 || !x || !target || !mask || !(lr > 0.0f))
        return mfail(mlp, DWOS_ERR_INVALID_ARG, "bad arguments");
    MK(cudaSetDevice(mlp->device), "cudaSetDevice");
    const float* in[3] = {x, target, mask};
    float* d[3];
    if (dwos_status s = stage(mlp, mem, 2 * (size_t)n, in, d, 3)) return s;
    if (dwos_status s = grads(mlp, n, d[0], d[1], d[2])) return s;
    mlp->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)mlp->step), c2 = 1.0f - powf(b2, (float)mlp->step);
    adam_kernel<<<(NP + 255) / 256, 256, 0, mlp->stream>>>(mlp->p, mlp->g, mlp->m, mlp->v, NP, lr, b1, b2, 1e-8f,
                                                           c1, c2);
    MK(cudaGetLastError(), "adam");
    convert_kernel<<<(H * H + 255) / 256, 256, 0, mlp->stream>>>(mlp->p, mlp->w);
    MK(cudaGetLastError(), "convert");
    if (loss) MK(cudaMemcpyAsync(loss, mlp->loss, sizeof(double),
                                 mem == DWOS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 mlp->stream), "copy loss");
    if (mem == DWOS_MEM_HOST) MK(cudaStreamSynchronize(mlp->stream), "synchronize");
    return DWOS_OK;
}

dwos_status dwos_mlp_eval(dwos_mlp* mlp, int n, const float* x, float* u, float* grad_u, float* q, int mem) {
    if (!mlp || n < 0 || (n > 0 && !x)) return mfail(mlp, DWOS_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return DWOS_OK;
    MK(cudaSetDevice(mlp->device), "cudaSetDevice");
    const float* in[1] = {x};
    float* d[1];
    if (dwos_status s = stage(mlp, mem, 2 * (size_t)n + 4 * (size_t)n, in, d, 1)) return s;
    float* du = u, *dg = grad_u, *dq = q;
    if (mem == DWOS_MEM_HOST) {   // outputs follow the staged input in scratch
        du = d[0] + 2 * (size_t)n;
        dg = du + n;
        dq = dg + 2 * (size_t)n;
    }
    eval_kernel<<<(n + 63) / 64, 64, 0, mlp->stream>>>(mlp->w, mlp->p, n, d[0], du, dg, dq);
    MK(cudaGetLastError(), "eval");
    if (mem == DWOS_MEM_HOST) {
        if (u) MK(cudaMemcpyAsync(u, du, sizeof(float) * n, cudaMemcpyDeviceToHost, mlp->stream), "copy");
        if (grad_u) MK(cudaMemcpyAsync(grad_u, dg, sizeof(float) * 2 * n, cudaMemcpyDeviceToHost, mlp->stream), "copy");
        if (q) MK(cudaMemcpyAsync(q, dq, sizeof(float) * n, cudaMemcpyDeviceToHost, mlp->stream), "copy");
        MK(cudaStreamSynchronize(mlp->stream), "synchronize");
    }
    return DWOS_OK;
}

}  // extern "C"
