// Control-variate network: features (x, y, sin pi x, sin pi y, sin pi (x+y))
// -> 4 x 64 tanh -> 8 linear outputs (0: u, 1: du/dn), trained and evaluated
// on the 5th-generation tensor cores.
//
// One persistent kernel (256 threads, one CTA per SM) walks over tiles of 128
// samples; sample row r is TMEM lane r, and threads r and r + 128 share it
// (warps w and w + 4 reach the same TMEM lane quarter): each takes half of the
// row's columns in the epilogues between the products.  Operands
// live in shared memory as BF16 in the canonical no-swizzle core-matrix
// layout (8 rows x 16 bytes per 128-byte core matrix), the products are
// tcgen05.mma (kind::f16, BF16 in, FP32 accumulate) issued by one thread and
// tracked by an mbarrier, and results come back with tcgen05.ld:
//   forward     D[128 x 64]  = A_{l-1}[128 x K] W_l^T        (A, B K-major)
//   backward    D[128 x 64]  = delta_l[128 x K] W_l           (B MN-major: W as stored)
//   weight grad dW_l[out x in+1] += delta_l^T A_{l-1}          (A, B MN-major)
// Each activation tile carries a constant-1 column, so the same product also
// accumulates the bias gradient.  Weight gradients stay in TMEM across all
// of a CTA's tiles and are written once per CTA; a second kernel sums the CTA
// partials in a fixed order (no atomics).  The BF16 weight image is copied
// into shared memory with one bulk asynchronous copy.  Evaluation runs the
// forward pass and the backward pass of output 0 (d u / d x) the same way.
//
// Flat FP32 parameter layout: W1 (64 x 16), b1 (64), W2 (64 x 64), b2, W3, b3,
// W4, b4, W5 (8 x 64), b5 (8); W[out][in] row-major.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "../../include/dwos.h"

namespace {

constexpr int H = 64;            // hidden width
constexpr int IN = 16;           // padded input width
constexpr int OUT = 8;           // output width
constexpr int OUTP = 16;         // output rows padded for the N = 16 product
constexpr int NP = DWOS_MLP_NPARAM;
constexpr int TILE = 128;        // samples per tile (the MMA's M)
constexpr int THREADS = 256;          // two threads per sample row
// offsets of W_l and b_l (l = 1..5) in the flat parameter vector
__host__ __device__ constexpr int off_w(int l) { return l == 1 ? 0 : 1088 + (l - 2) * 4160; }
__host__ __device__ constexpr int off_b(int l) { return l == 1 ? 1024 : (l == 5 ? 14080 : 1088 + (l - 2) * 4160 + 4096); }
static_assert(off_b(5) + 8 == DWOS_MLP_NPARAM, "parameter layout");

// Element offset of (row, col) in a BF16 tile of C columns, canonical
// no-swizzle layout: core matrix (row / 8, col / 8) is 64 contiguous elements,
// row-major inside (16 bytes per row); core matrices of one 8-row group are
// consecutive along the columns (128 bytes apart), groups are C * 16 bytes apart.
__host__ __device__ constexpr int core_off(int row, int col, int C) {
    return ((row >> 3) * (C >> 3) + (col >> 3)) * 64 + (row & 7) * 8 + (col & 7);
}

// BF16 weight image, in the shared-memory layout (one bulk copy).
struct WImage {
    __nv_bfloat16 w1[H * IN];        // 64 x 16
    __nv_bfloat16 w2[H * H], w3[H * H], w4[H * H];
    __nv_bfloat16 w5[OUTP * H];      // 16 x 64, rows 8..15 zero
};
static_assert(sizeof(WImage) % 16 == 0, "bulk copy size");

constexpr int C0 = 32;           // input tile: 16 features, the constant 1 at column 16, zeros
constexpr int CA = 80;           // hidden tiles: 64 activations, the constant 1 at column 64, zeros
constexpr int CD = 128;          // delta tile: 64 (or 16) deltas, zeros (rows of the M = 128 weight-gradient product)

struct __align__(1024) Smem {
    WImage w;                                   // 28672 B
    __nv_bfloat16 a0[TILE * C0];                // 8 KB
    __nv_bfloat16 a[4][TILE * CA];              // 4 x 20 KB
    __nv_bfloat16 d[TILE * CD];                 // 32 KB
    float bias[4 * H + OUT];
    unsigned long long bar_load, bar_mma;
    uint32_t tmem_base;
    int fail;
};

// TMEM columns (512 allocated)
constexpr uint32_t T_SCR = 0;                   // 64: forward / backward products
// dW_l with its bias column (32, 80, 80, 80, 80 columns) for l = 1..5
__host__ __device__ constexpr uint32_t t_dw(int l) { return l == 1 ? 64u : 96u + 80u * (uint32_t)(l - 2); }
constexpr uint32_t TMEM_COLS = 512;

// ---- PTX wrappers -------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B BF16 (bits
// 7-9, 10-12 = 1), A / B major-ness (bits 15, 16: 0 K-major, 1 MN-major),
// N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn, bool b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Shared-memory matrix descriptor, no swizzle: start address, leading-dimension
// byte offset (between core matrices along K for K-major operands, along the
// 8-element K groups for MN-major ones), stride byte offset (the other
// direction), all >> 4; bit 46 set (descriptor version of this architecture).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// K-major view of a tile with C columns, K step ks (16 columns)
__device__ __forceinline__ uint64_t kmajor(const __nv_bfloat16* tile, int C, int ks) {
    return sdesc(smem_u32(tile) + ks * 256, 128, (C / 8) * 128);
}
// MN-major view of a tile with C columns (MN = columns, K = rows), K step ks (16 rows)
__device__ __forceinline__ uint64_t mnmajor(const __nv_bfloat16* tile, int C, int ks) {
    return sdesc(smem_u32(tile) + ks * 2 * (C / 8) * 128, (C / 8) * 128, 128);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait: false if the phase never completed within `polls` tries.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, int polls = 1 << 24) {
    for (int i = 0; i < polls; ++i)
        if (bar_try(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
// write 8 values (one core-matrix row) of row r, column chunk cc of a tile with C columns
__device__ __forceinline__ void put8(__nv_bfloat16* tile, int C, int r, int cc, const float* v) {
    uint4 q;
    q.x = pack2(v[0], v[1]); q.y = pack2(v[2], v[3]); q.z = pack2(v[4], v[5]); q.w = pack2(v[6], v[7]);
    *reinterpret_cast<uint4*>(tile + core_off(r, cc * 8, C)) = q;
}
__device__ __forceinline__ void get8(const __nv_bfloat16* tile, int C, int r, int cc, float* v) {
    const uint4 q = *reinterpret_cast<const uint4*>(tile + core_off(r, cc * 8, C));
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&w[i]);
        v[2 * i] = __low2float(b);
        v[2 * i + 1] = __high2float(b);
    }
}

__device__ __forceinline__ void feats(float x, float y, float* f) {
    f[0] = x;
    f[1] = y;
    f[2] = sinpif(x);
    f[3] = sinpif(y);
    f[4] = sinpif(x + y);
}

enum Mode { kTrain = 0, kEval = 1 };

// mode kTrain: masked-MSE loss (sum over this CTA's samples, FP64, one atomic
// per warp) and the CTA's gradient partial (NP floats at part + blockIdx.x * NP).
// mode kEval: u, d u / d (x, y) and du/dn per sample.
template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
    mlp_kernel(const WImage* __restrict__ wimg, const float* __restrict__ params, int n,
               const float* __restrict__ x, const float* __restrict__ target, const float* __restrict__ mask,
               float* __restrict__ part, double* __restrict__ loss, float* __restrict__ u_out,
               float* __restrict__ g_out, float* __restrict__ q_out, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char raw[];
    Smem& S = *reinterpret_cast<Smem*>(raw);
    const int tid = threadIdx.x;
    const int r = tid & (TILE - 1);            // sample row and TMEM lane
    const int half = tid >> 7;                 // which half of the row's columns this thread takes
    const int warp = tid >> 5;
    const uint32_t bar_load = smem_u32(&S.bar_load), bar_mma = smem_u32(&S.bar_mma);
    if (tid == 0) {
        bar_init(bar_load, 1);
        bar_init(bar_mma, 1);
        S.fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&S.tmem_base)), "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // constants: biases; zero the columns of the tiles that no tile overwrites
    for (int i = tid; i < 4 * H + OUT; i += THREADS)
        S.bias[i] = params[i < 4 * H ? off_b(1 + i / H) + i % H : off_b(5) + (i - 4 * H)];
    {
        const float z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        const float one[8] = {1, 0, 0, 0, 0, 0, 0, 0};
        if (half == 0) {
            put8(S.a0, C0, r, 2, one);
            put8(S.a0, C0, r, 3, z);
            for (int l = 0; l < 4; ++l) {
                put8(S.a[l], CA, r, 8, one);
                put8(S.a[l], CA, r, 9, z);
            }
        }
        for (int cc = half * (CD / 16); cc < (half + 1) * (CD / 16); ++cc) put8(S.d, CD, r, cc, z);
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_base;
    const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);   // this warp's TMEM lane quarter
    if (tid == 0) {
        bar_expect_tx(bar_load, sizeof(WImage));
        bulk_g2s(smem_u32(&S.w), wimg, sizeof(WImage), bar_load);
    }
    bool ok = bar_wait(bar_load, 0);
    ok = !__syncthreads_or(!ok);
    uint32_t phase = 0;
    const __nv_bfloat16* W[6] = {nullptr, S.w.w1, S.w.w2, S.w.w3, S.w.w4, S.w.w5};
    const int CW[6] = {0, IN, H, H, H, H};     // columns of W_l (its K in the forward product)
    const float inv_n = 1.0f / (float)n;
    float loss_acc = 0.0f;
    const int n_tiles = (n + TILE - 1) / TILE;

    // thread 0 commits the issued products; everyone waits; false if any wait failed
    auto sync_mma = [&]() -> bool {
        if (tid == 0) mma_commit(bar_mma);
        const bool got = bar_wait(bar_mma, phase);
        phase ^= 1u;
        fence_after();
        return !__syncthreads_or(!got);
    };
    auto publish = [&]() {     // smem written by the threads -> visible to the next products
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
    };

    int tiles_done = 0;
    for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x, ++tiles_done) {
        const int s = tile * TILE + r;
        const bool valid = s < n;
        float px = 0.0f, py = 0.0f;
        if (valid) { px = x[2 * s]; py = x[2 * s + 1]; }
        if (half == 0) {
            float f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (valid) feats(px, py, f);
            const float z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            put8(S.a0, C0, r, 0, f);
            put8(S.a0, C0, r, 1, z);
        }
        publish();
        // ---- forward: four tanh layers
        for (int l = 1; l <= 4 && ok; ++l) {
            const __nv_bfloat16* A = l == 1 ? S.a0 : S.a[l - 2];
            const int CAin = l == 1 ? C0 : CA;
            if (tid == 0) {
                fence_after();
                for (int ks = 0; ks < CW[l] / 16; ++ks)
                    mma(tmem + T_SCR, kmajor(A, CAin, ks), kmajor(W[l], CW[l], ks), idesc_bf16(128, 64, false, false),
                        ks > 0 ? 1u : 0u);
            }
            ok = sync_mma();
            if (!ok) break;
            for (int c16 = 2 * half; c16 < 2 * half + 2; ++c16) {
                float v[16];
                tmem_ld16(lane_addr + T_SCR + 16 * c16, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = tanhf(v[i] + S.bias[(l - 1) * H + 16 * c16 + i]);
                put8(S.a[l - 1], CA, r, 2 * c16, v);
                put8(S.a[l - 1], CA, r, 2 * c16 + 1, v + 8);
            }
            publish();
        }
        if (!ok) break;
        // ---- output layer
        if (tid == 0) {
            fence_after();
            for (int ks = 0; ks < 4; ++ks)
                mma(tmem + T_SCR, kmajor(S.a[3], CA, ks), kmajor(S.w.w5, H, ks), idesc_bf16(128, 16, false, false),
                    ks > 0 ? 1u : 0u);
        }
        ok = sync_mma();
        if (!ok) break;
        if (half == 0) {
            float o[16];
            tmem_ld16(lane_addr + T_SCR, o);
            float d5[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) d5[i] = 0.0f;
            if (MODE == kTrain) {
                if (valid)
                    for (int k = 0; k < 2; ++k) {
                        const float e = mask[2 * s + k] * (o[k] + S.bias[4 * H + k] - target[2 * s + k]);
                        loss_acc += e * e;
                        d5[k] = 2.0f * e * inv_n;
                    }
            } else {
                if (valid) {
                    if (u_out) u_out[s] = o[0] + S.bias[4 * H];
                    if (q_out) q_out[s] = o[1] + S.bias[4 * H + 1];
                }
                d5[0] = 1.0f;        // d u / d out
            }
            put8(S.d, CD, r, 0, d5);
            put8(S.d, CD, r, 1, d5 + 8);
        }
        publish();
        // ---- backward: weight gradients (training) and the deltas
        for (int l = 5; l >= 1 && ok; --l) {
            const __nv_bfloat16* Ain = l == 1 ? S.a0 : S.a[l - 2];
            const int CAin = l == 1 ? C0 : CA;
            const bool delta_product = l > 1 || MODE == kEval;
            if (tid == 0) {
                fence_after();
                if (MODE == kTrain)
                    for (int ks = 0; ks < TILE / 16; ++ks)
                        mma(tmem + t_dw(l), mnmajor(S.d, CD, ks), mnmajor(Ain, CAin, ks),
                            idesc_bf16(128, CAin, true, true), (tiles_done > 0 || ks > 0) ? 1u : 0u);
                if (delta_product) {
                    const int kout = l == 5 ? OUTP : H;  // K of the product: layer l's outputs
                    const int nin = l == 1 ? IN : H;     // N: its inputs
                    for (int ks = 0; ks < kout / 16; ++ks)
                        mma(tmem + T_SCR, kmajor(S.d, CD, ks), mnmajor(W[l], CW[l], ks),
                            idesc_bf16(128, nin, false, true), ks > 0 ? 1u : 0u);
                }
            }
            ok = sync_mma();
            if (!ok) break;
            if (l > 1) {
                // delta_{l-1} = (delta_l W_l) * (1 - a_{l-1}^2), a as stored (BF16)
                for (int c16 = 2 * half; c16 < 2 * half + 2; ++c16) {
                    float v[16], a[16];
                    tmem_ld16(lane_addr + T_SCR + 16 * c16, v);
                    get8(S.a[l - 2], CA, r, 2 * c16, a);
                    get8(S.a[l - 2], CA, r, 2 * c16 + 1, a + 8);
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] *= 1.0f - a[i] * a[i];
                    put8(S.d, CD, r, 2 * c16, v);
                    put8(S.d, CD, r, 2 * c16 + 1, v + 8);
                }
                publish();
            } else if (MODE == kEval) {
                float df[16];
                if (half == 0) tmem_ld16(lane_addr + T_SCR, df);       // d u / d features
                if (half == 0 && valid && g_out) {
                    const float c0 = 3.14159265358979f * cospif(px), c1 = 3.14159265358979f * cospif(py);
                    const float c01 = 3.14159265358979f * cospif(px + py);
                    g_out[2 * s] = df[0] + df[2] * c0 + df[4] * c01;
                    g_out[2 * s + 1] = df[1] + df[3] * c1 + df[4] * c01;
                }
                fence_before();
                __syncthreads();
                fence_after();
            }
        }
    }

    if (MODE == kTrain && ok) {
        for (int off = 16; off > 0; off >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
        if ((tid & 31) == 0 && loss_acc != 0.0f) atomicAdd(loss, (double)loss_acc * (double)inv_n);
        // the CTA's weight and bias gradients: rows (outputs) are TMEM lanes 0..63
        float* P = part + (size_t)blockIdx.x * NP;
        for (int l = 1; l <= 5; ++l) {
            const int outs = l == 5 ? OUT : H, ins = l == 1 ? IN : H;
            const int ncol = l == 1 ? C0 : CA;
            for (int c16 = half; c16 < ncol / 16; c16 += 2) {
                float v[16];
                tmem_ld16(lane_addr + t_dw(l) + 16 * c16, v);     // warp-wide: every warp loads
                if (r < outs)
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int c = 16 * c16 + i;
                        if (c < ins) P[off_w(l) + r * ins + c] = v[i];
                        else if (c == ins) P[off_b(l) + r] = v[i];
                    }
            }
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS));
    if (tid == 0 && !ok) atomicOr(err, 1);
}

// The failure path of the bounded wait, without a fault: thread 0 initialises an
// mbarrier that nothing ever arrives at (no copy or product is issued, so nothing
// is in flight), every thread waits on it with the training kernel's bar_wait and
// gives up after `polls` tries, and the give-up is reported through the same flag.
__global__ void wait_probe_kernel(int polls, int* __restrict__ err) {
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        bar_init(b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool got = bar_wait(b, 0, polls);
    if (!__syncthreads_or(!got)) return;
    if (threadIdx.x == 0) atomicOr(err, 1);
}

// Sum of the CTA partials, in CTA order (deterministic).
__global__ void reduce_parts_kernel(const float* __restrict__ part, int n_parts, float* __restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    float s = 0.0f;
    for (int c = 0; c < n_parts; ++c) s += part[(size_t)c * NP + i];
    grad[i] = s;
}

// BF16 weight image in the shared-memory layout.
__global__ void convert_kernel(const float* __restrict__ p, WImage* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < H * IN) {
        const int o = i / IN, c = i % IN;
        w->w1[core_off(o, c, IN)] = __float2bfloat16_rn(p[off_w(1) + i]);
    }
    if (i < H * H) {
        const int o = i / H, c = i % H;
        w->w2[core_off(o, c, H)] = __float2bfloat16_rn(p[off_w(2) + i]);
        w->w3[core_off(o, c, H)] = __float2bfloat16_rn(p[off_w(3) + i]);
        w->w4[core_off(o, c, H)] = __float2bfloat16_rn(p[off_w(4) + i]);
    }
    if (i < OUTP * H) {
        const int o = i / H, c = i % H;
        w->w5[core_off(o, c, H)] = __float2bfloat16_rn(o < OUT ? p[off_w(5) + o * H + c] : 0.0f);
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
    WImage* w = nullptr;         // BF16 weight image
    float* part = nullptr;       // per-CTA gradient partials (n_sm x NP)
    int* dflag = nullptr;        // device flag: a bounded wait ran out
    int n_sm = 0;
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

int grid_for(const dwos_mlp* mlp, int n) {
    const int tiles = (n + TILE - 1) / TILE;
    return tiles < mlp->n_sm ? tiles : mlp->n_sm;
}

dwos_status check_err(dwos_mlp* mlp) {
    int e = 0;
    MK(cudaMemcpyAsync(&e, mlp->dflag, sizeof(int), cudaMemcpyDeviceToHost, mlp->stream), "read flag");
    MK(cudaStreamSynchronize(mlp->stream), "synchronize");
    if (e) {   // reported once: the next call starts with a clear flag
        MK(cudaMemsetAsync(mlp->dflag, 0, sizeof(int), mlp->stream), "reset flag");
        return mfail(mlp, DWOS_ERR_TIMEOUT, "a bounded wait on the tensor-core kernel's mbarrier ran out");
    }
    return DWOS_OK;
}

dwos_status grads(dwos_mlp* mlp, int n, const float* x, const float* t, const float* mk) {
    MK(cudaMemsetAsync(mlp->loss, 0, sizeof(double), mlp->stream), "zero loss");
    const int grid = grid_for(mlp, n);
    mlp_kernel<kTrain><<<grid, THREADS, sizeof(Smem), mlp->stream>>>(mlp->w, mlp->p, n, x, t, mk, mlp->part,
                                                                     mlp->loss, nullptr, nullptr, nullptr, mlp->dflag);
    MK(cudaGetLastError(), "train kernel");
    reduce_parts_kernel<<<(NP + 255) / 256, 256, 0, mlp->stream>>>(mlp->part, grid, mlp->g);
    MK(cudaGetLastError(), "reduce");
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
    if (e == cudaSuccess) e = cudaMalloc(&mlp->w, sizeof(WImage));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mlp->n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&mlp->part, sizeof(float) * NP * (size_t)(mlp->n_sm > 0 ? mlp->n_sm : 1));
    if (e == cudaSuccess) e = cudaMalloc(&mlp->dflag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(mlp->dflag, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(mlp->w, 0, sizeof(WImage));
    if (e == cudaSuccess) e = cudaMemset(mlp->p, 0, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMemset(mlp->m, 0, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMemset(mlp->v, 0, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(mlp_kernel<kTrain>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)sizeof(Smem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(mlp_kernel<kEval>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
                    (void*)mlp->scratch, (void*)mlp->part, (void*)mlp->dflag})
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
    if (mem == DWOS_MEM_HOST) return check_err(mlp);
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
    if (mem == DWOS_MEM_HOST) return check_err(mlp);
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
    mlp_kernel<kEval><<<grid_for(mlp, n), THREADS, sizeof(Smem), mlp->stream>>>(
        mlp->w, mlp->p, n, d[0], nullptr, nullptr, nullptr, nullptr, du, dg, dq, mlp->dflag);
    MK(cudaGetLastError(), "eval");
    if (mem == DWOS_MEM_HOST) {
        if (u) MK(cudaMemcpyAsync(u, du, sizeof(float) * n, cudaMemcpyDeviceToHost, mlp->stream), "copy");
        if (grad_u) MK(cudaMemcpyAsync(grad_u, dg, sizeof(float) * 2 * n, cudaMemcpyDeviceToHost, mlp->stream), "copy");
        if (q) MK(cudaMemcpyAsync(q, dq, sizeof(float) * n, cudaMemcpyDeviceToHost, mlp->stream), "copy");
        return check_err(mlp);
    }
    return DWOS_OK;
}

dwos_status dwos_mlp_sync(dwos_mlp* mlp) {
    if (!mlp) return mfail(nullptr, DWOS_ERR_INVALID_ARG, "mlp is NULL");
    MK(cudaSetDevice(mlp->device), "cudaSetDevice");
    return check_err(mlp);
}

dwos_status dwos_mlp_wait_probe(dwos_mlp* mlp, int polls) {
    if (!mlp) return mfail(nullptr, DWOS_ERR_INVALID_ARG, "mlp is NULL");
    if (polls < 1 || polls > (1 << 24)) return mfail(mlp, DWOS_ERR_INVALID_ARG, "polls must be in [1, 2^24]");
    MK(cudaSetDevice(mlp->device), "cudaSetDevice");
    if (dwos_status s = check_err(mlp)) return s;     // earlier work first
    wait_probe_kernel<<<1, 128, 0, mlp->stream>>>(polls, mlp->dflag);
    MK(cudaGetLastError(), "wait probe");
    return check_err(mlp);
}

}  // extern "C"
