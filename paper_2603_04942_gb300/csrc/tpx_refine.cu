// tpx_refine.cu -- the learned overlap refiner (not in the paper; its
// multi-hit discussion, Sec. VII.B, motivates it): a cluster larger than a
// few pixels may hold two particles. Its 9x9 patch of ToT and relative ToA
// around the rounded centroid goes through a small multilayer perceptron that
// predicts one or two particles and their positions; below a confidence
// threshold the plain centroid (Sec. V.C) stands.
//
//   patches : clusters with more than `min_pixels` pixels; per packet of such
//             a cluster one cell of its patch (the brighter pixel wins a
//             shared cell, ties to the later one).
//   MLP     : 162 inputs -> H (ReLU) -> H (ReLU) -> 6 outputs: two logits
//             (one / two particles) and two offsets (dx, dy) per particle,
//             in pixels from the patch centre. fp32 tiled GEMMs (a dense
//             contraction), bias/ReLU in the epilogue.
//   training: softmax cross-entropy on the count, squared error on the
//             offsets of the true particles, Adam; one call per minibatch.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "tpx.h"
#include "tpx_common.cuh"
#include "tpx_ctx.h"

namespace tpxr {

using namespace tpxk;

constexpr int PS = 9;                 // patch side
constexpr int PC = PS * PS;           // cells per channel
constexpr int NIN = 2 * PC;           // MLP inputs
constexpr int NOUT = 6;               // logits (2) + offsets (4)

inline bool ck(cudaError_t e, int line = __builtin_LINE()) {
    if (e == cudaSuccess) return false;
    if (std::getenv("TPX_DEBUG")) std::fprintf(stderr, "tpx_refine.cu:%d: %s\n", line, cudaGetErrorString(e));
    return true;
}
inline unsigned grid_for(long long n, int bt = 256) {
    long long g = (n + bt - 1) / bt;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)g;
}

// ---------------------------------------------------------------- patches
__global__ void k_sel_flags(const tpx_record *cl, long long ncl, int min_px, unsigned *f) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncl; i += (long long)gridDim.x * blockDim.x)
        f[i] = cl[i].n > min_px ? 1u : 0u;
}
// exclusive scan in three steps: per-block sums, one block over them, add
constexpr int SB = 1024;
__global__ void k_scan_local(const unsigned *in, unsigned *out, long long n, unsigned *bsum) {
    __shared__ unsigned s[SB];
    const long long i = blockIdx.x * (long long)SB + threadIdx.x;
    const unsigned v = i < n ? in[i] : 0u;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < SB; o <<= 1) {
        const unsigned u = threadIdx.x >= o ? s[threadIdx.x - o] : 0u;
        __syncthreads();
        s[threadIdx.x] += u;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;
    if (threadIdx.x == SB - 1) bsum[blockIdx.x] = s[SB - 1];
}
// exclusive scan of the block sums by one block, SB at a time
__global__ void k_scan_sums(unsigned *bsum, long long nb, long long *total) {
    __shared__ unsigned s[SB];
    __shared__ unsigned carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b0 = 0; b0 < nb; b0 += SB) {
        const long long b = b0 + threadIdx.x;
        const unsigned v = b < nb ? bsum[b] : 0u;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < SB; o <<= 1) {
            const unsigned u = threadIdx.x >= o ? s[threadIdx.x - o] : 0u;
            __syncthreads();
            s[threadIdx.x] += u;
            __syncthreads();
        }
        if (b < nb) bsum[b] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == SB - 1) carry += s[SB - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}
__global__ void k_scan_add(unsigned *out, long long n, const unsigned *bsum) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] += bsum[i / SB];
}
__global__ void k_select(const uint64_t *pk, const tpx_record *cl, long long ncl, const unsigned *f, const unsigned *off,
                         long long cap, long long base, long long n, long long *sel, int *centre, int *slot_of_root) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncl; i += (long long)gridDim.x * blockDim.x) {
        if (!f[i]) continue;
        const long long s = off[i];
        if (s >= cap) continue;
        sel[s] = i;
        const long long r = cl[i].label - base;
        const tpx_record &c = cl[i];
        int cx = 0, cy = 0;
        if (c.s_tot > 0) {   // the centroid rounded half up, exactly: floor((2 s_x + s_tot) / (2 s_tot))
            cx = (int)((2 * c.s_x + c.s_tot) / (2 * c.s_tot));
            cy = (int)((2 * c.s_y + c.s_tot) / (2 * c.s_tot));
        } else if (r >= 0 && r < n) {   // no charge: the earliest pixel
            cx = pix_x(pk[r]);
            cy = pix_y(pk[r]);
        }
        centre[2 * s] = cx;
        centre[2 * s + 1] = cy;
        if (r >= 0 && r < n) slot_of_root[r] = (int)s;   // else not a record of these packets: an empty patch
    }
}
__global__ void k_fill_i32(int *p, long long n, int v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) p[i] = v;
}
// the brighter pixel of a shared cell wins (ties: the later one)
__global__ void k_patch_keys(const uint64_t *pk, long long n, long long base, const long long *labels,
                             const int *slot_of_root, const int *centre, unsigned long long *key) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const long long L = labels[q] - base;
        if (labels[q] < 0 || L < 0 || L >= n) continue;
        const int s = slot_of_root[L];
        if (s < 0) continue;
        const uint64_t w = pk[q];
        const int dx = pix_x(w) - centre[2 * s] + PS / 2, dy = pix_y(w) - centre[2 * s + 1] + PS / 2;
        if (dx < 0 || dx >= PS || dy < 0 || dy >= PS) continue;
        const unsigned long long k = ((unsigned long long)(pix_tot(w) + 1) << 40) | (unsigned long long)q;
        atomicMax(&key[(long long)s * PC + dy * PS + dx], k);
    }
}
// channel 0: ToT / 1023 rounded to bf16; channel 1: ToA relative to the
// cluster's earliest pixel, in units of 32 ticks (50 ns), clamped to [-8, 8],
// rounded to fp16 (exact: multiples of 1/32 below 8); empty cells 0
template <typename OutT>
__global__ void k_patch_fill(const uint64_t *pk, long long base, const tpx_record *cl, const long long *sel,
                             const unsigned long long *key, long long ns, OutT *patch) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ns * PC; c += (long long)gridDim.x * blockDim.x) {
        const long long s = c / PC;
        const int cell = (int)(c % PC);
        float tot = 0.f, rel = 0.f;
        const unsigned long long k = key[c];
        if (k) {
            const long long q = (long long)(k & ((1ull << 40) - 1));
            const uint64_t w = pk[q];
            const uint64_t w0 = pk[cl[sel[s]].label - base];   // in range: the key came from this cluster
            long long d = (pix_raw(w) - pix_raw(w0)) & (kPixPeriod - 1);
            if (d >= kPixPeriod / 2) d -= kPixPeriod;   // the signed difference, wrap-safe
            // the patch precisions: ToT in bf16, relative ToA in fp16 (held widened to fp32)
            tot = __bfloat162float(__float2bfloat16_rn((float)pix_tot(w) / 1023.f));
            rel = __half2float(__float2half_rn(fminf(8.f, fmaxf(-8.f, (float)d / 32.f))));
        }
        if (sizeof(OutT) == 4) {
            patch[s * NIN + cell] = tot;
            patch[s * NIN + PC + cell] = rel;
        } else {   // exact in bf16 as well
            reinterpret_cast<__nv_bfloat16 *>(patch)[s * NIN + cell] = __float2bfloat16_rn(tot);
            reinterpret_cast<__nv_bfloat16 *>(patch)[s * NIN + PC + cell] = __float2bfloat16_rn(rel);
        }
    }
}

// ---------------------------------------------------------------- GEMM
// C[M x N] = op(A)[M x K] * op(B)[K x N] (+ bias[N]) (ReLU), with op given
// by strides: A(i, k) = A[i * sam + k * sak], B(k, j) = B[k * sbk + j * sbn].
// 64 x 64 tiles, 256 threads, 4 x 4 outputs per thread.
constexpr int TM = 64, TN = 64, TK = 16;
__global__ void __launch_bounds__(256) k_gemm(const float *A, long long sam, long long sak, const float *B,
                                              long long sbk, long long sbn, float *C, long long ldc, int M, int N,
                                              int K, const float *bias, int relu, int accumulate) {
    __shared__ float As[TK][TM + 4];
    __shared__ float Bs[TK][TN + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += TK) {
        // consecutive threads walk the operand's unit-stride dimension (coalesced loads)
        for (int t = threadIdx.x; t < TK * TM; t += 256) {
            const int kk = sak == 1 ? t % TK : t / TM, ii = sak == 1 ? t / TK : t % TM;
            const int i = i0 + ii, k = k0 + kk;
            As[kk][ii] = (i < M && k < K) ? A[i * sam + k * sak] : 0.f;
        }
        for (int t = threadIdx.x; t < TK * TN; t += 256) {
            const int kk = sbk == 1 ? t % TK : t / TN, jj = sbk == 1 ? t / TK : t % TN;
            const int j = j0 + jj, k = k0 + kk;
            Bs[kk][jj] = (j < N && k < K) ? B[k * sbk + j * sbn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
            for (int r = 0; r < 4; ++r) b[r] = Bs[kk][tx * 4 + r];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(a[r], b[q], acc[r][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + ty * 4 + r, j = j0 + tx * 4 + q;
            if (i >= M || j >= N) continue;
            float v = acc[r][q];
            if (accumulate) v += C[(long long)i * ldc + j];
            if (bias) v += bias[j];
            if (relu) v = fmaxf(v, 0.f);
            C[(long long)i * ldc + j] = v;
        }
}
void gemm(cudaStream_t s, const float *A, long long sam, long long sak, const float *B, long long sbk, long long sbn,
          float *C, long long ldc, int M, int N, int K, const float *bias, bool relu, bool accumulate = false) {
    dim3 g((N + TN - 1) / TN, (M + TM - 1) / TM);
    k_gemm<<<g, 256, 0, s>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, bias, relu ? 1 : 0, accumulate ? 1 : 0);
}

// parameter layout (floats): W1[NIN x H], b1[H], W2[H x H], b2[H], W3[H x NOUT], b3[NOUT]
struct Layout {
    int h;
    long long w1, b1, w2, b2, w3, b3, total;
    __host__ __device__ explicit Layout(int hidden) : h(hidden) {
        w1 = 0; b1 = w1 + (long long)NIN * h; w2 = b1 + h; b2 = w2 + (long long)h * h; w3 = b2 + h;
        b3 = w3 + (long long)h * NOUT; total = b3 + NOUT;
    }
};

// loss of a minibatch and its gradient at the outputs: y = [count(1|2), dx1, dy1, dx2, dy2]
__global__ void k_loss(const float *out, const float *y, int n, float w_off, float *dout, float *loss) {
    __shared__ float part[256];
    float l = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float *o = out + (long long)i * NOUT;
        const float *t = y + (long long)i * 5;
        const int two = t[0] > 1.5f;
        const float m = fmaxf(o[0], o[1]);
        const float e0 = __expf(o[0] - m), e1 = __expf(o[1] - m), z = e0 + e1;
        const float p1 = e1 / z;
        l += -((two ? o[1] : o[0]) - m - __logf(z));
        float *g = dout + (long long)i * NOUT;
        const float inv = 1.f / (float)n;
        g[0] = ((1.f - p1) - (two ? 0.f : 1.f)) * inv;
        g[1] = (p1 - (two ? 1.f : 0.f)) * inv;
        for (int k = 0; k < 4; ++k) {
            const bool used = k < 2 || two;
            const float d = used ? o[2 + k] - t[1 + k] : 0.f;
            l += 0.5f * w_off * d * d;
            g[2 + k] = w_off * d * inv;
        }
    }
    part[threadIdx.x] = l;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, part[0] / (float)n);
}
// dZ = dA where the forward activation was positive (ReLU)
__global__ void k_relu_back(float *d, const float *act, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (act[i] <= 0.f) d[i] = 0.f;
}
// bias gradient: column sums of dZ [n x m]
__global__ void k_colsum(const float *d, int n, int m, float *g) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int i = 0; i < n; ++i) s += d[(long long)i * m + j];
        g[j] = s;
    }
}
__global__ void k_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// refined hits: per patch the network's two positions when it is confident of
// two particles, else the plain centroid (k = 1 when it is confident of one,
// k = 0 when of neither). p(two) >= thr  <=>  logit margin o1 - o0 >= log(thr / (1 - thr)),
// decided on the fp32 margin so the count is exact, not at the mercy of exp.
__global__ void k_decide(const float *out, const tpx_record *cl, const long long *sel, const int *centre, long long n,
                         float lt, float *hits /* n x 5: n_hits, x1, y1, x2, y2 */) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const float *o = out + s * NOUT;
        const float margin = o[1] - o[0];
        const float cx = (float)centre[2 * s], cy = (float)centre[2 * s + 1];
        float *h = hits + s * 5;
        if (margin >= lt) {   // two particles: the network's positions
            h[0] = 2.f; h[1] = cx + o[2]; h[2] = cy + o[3]; h[3] = cx + o[4]; h[4] = cy + o[5];
        } else {              // one particle (1), or not confident (0): the plain centroid
            const tpx_record &r = cl[sel[s]];
            h[0] = -margin >= lt ? 1.f : 0.f; h[1] = (float)r.x; h[2] = (float)r.y; h[3] = 0.f; h[4] = 0.f;
        }
    }
}

// ---------------------------------------------------------------- bf16 inference
// The whole network in one persistent kernel on the tensor cores
// (mma.sync m16n8k16, bf16 operands, fp32 accumulation). Each warp owns 16
// patches and carries them through the three layers: the fp32 accumulator
// fragment of one layer, after bias and ReLU, is exactly the bf16 A-operand
// fragment of the next (row g = lane / 4 and column pair 2 (lane % 4) of
// n-tile j are row g, k pair of k-step j / 2), so activations never leave
// registers. The weights, transposed to [n][k] bf16 by tpx_refiner_pack, sit
// in shared memory for the kernel's lifetime; patches stream from global
// memory as fp32 pairs (8-byte loads; a row's 4 lanes read one 32-byte
// sector) and are rounded to bf16 (exact for the patch precisions).
constexpr int K1P = 176;                       // 162 inputs padded to 11 k-steps
constexpr int S1 = K1P + 8;                    // smem row stride of W1t (92 words: conflict-free)
template <int H> struct MlpGeo {
    static constexpr int S2 = H + 8;           // smem row stride of W2t / W3t
    static constexpr int NT = H / 8;           // n-tiles of a hidden layer
    static constexpr int KS = H / 16;          // k-steps over a hidden layer
    static constexpr size_t w1 = 0, w2 = w1 + (size_t)H * K1P, w3 = w2 + (size_t)H * H, wend = w3 + (size_t)8 * H;
    static constexpr size_t packed_bytes = ((wend * 2 + 15) / 16) * 16 + (size_t)(2 * H + 8) * 4;
    static constexpr size_t smem = (size_t)H * S1 * 2 + (size_t)H * S2 * 2 + (size_t)8 * S2 * 2 + (size_t)(2 * H + 8) * 4;
};
inline size_t packed_bias_off(size_t wend) { return ((wend * 2 + 15) / 16) * 16; }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (lower k) in the low half
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// fp32 parameters -> W1t [H][176], W2t [H][H], W3t [8][H] bf16 (zero padded),
// then b1, b2, b3 (padded to 8) fp32
template <int H>
__global__ void k_pack(const float *P, uint16_t *wt, float *bias) {
    using G = MlpGeo<H>;
    const Layout L(H);
    const long long total = (long long)G::wend + 2 * H + 8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        if (i >= (long long)G::wend) {
            const int b = (int)(i - G::wend);
            bias[b] = b < H ? P[L.b1 + b] : b < 2 * H ? P[L.b2 + b - H] : (b - 2 * H < NOUT ? P[L.b3 + b - 2 * H] : 0.f);
            continue;
        }
        float v = 0.f;
        if (i < (long long)G::w2) {
            const int j = (int)(i / K1P), k = (int)(i % K1P);
            if (k < NIN) v = P[L.w1 + (long long)k * H + j];
        } else if (i < (long long)G::w3) {
            const long long r = i - G::w2;
            const int j = (int)(r / H), k = (int)(r % H);
            v = P[L.w2 + (long long)k * H + j];
        } else {
            const long long r = i - G::w3;
            const int j = (int)(r / H), k = (int)(r % H);
            if (j < NOUT) v = P[L.w3 + (long long)k * NOUT + j];
        }
        __nv_bfloat16 b = __float2bfloat16_rn(v);
        wt[i] = *reinterpret_cast<uint16_t *>(&b);
    }
}

// hidden layer epilogue: bias was the accumulator's start; ReLU, round to
// bf16 and regroup n-tile pairs into next-layer A fragments
template <int NT>
__device__ __forceinline__ void to_frags(const float (&acc)[NT][4], uint32_t (&a)[NT / 2][4]) {
#pragma unroll
    for (int s = 0; s < NT / 2; ++s) {
        a[s][0] = pack_bf16(fmaxf(acc[2 * s][0], 0.f), fmaxf(acc[2 * s][1], 0.f));
        a[s][1] = pack_bf16(fmaxf(acc[2 * s][2], 0.f), fmaxf(acc[2 * s][3], 0.f));
        a[s][2] = pack_bf16(fmaxf(acc[2 * s + 1][0], 0.f), fmaxf(acc[2 * s + 1][1], 0.f));
        a[s][3] = pack_bf16(fmaxf(acc[2 * s + 1][2], 0.f), fmaxf(acc[2 * s + 1][3], 0.f));
    }
}

template <int H>
__global__ void __launch_bounds__(256, 1) k_mlp_bf16(const float *__restrict__ x, long long n,
                                                      const uint16_t *__restrict__ wt, const float *__restrict__ bias,
                                                      float *__restrict__ out) {
    using G = MlpGeo<H>;
    constexpr int NT = G::NT, S2 = G::S2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t *W1s = reinterpret_cast<uint16_t *>(smem_raw);
    uint16_t *W2s = W1s + H * S1;
    uint16_t *W3s = W2s + H * S2;
    float *Bs = reinterpret_cast<float *>(W3s + 8 * S2);
    // weights into shared memory, 16 bytes at a time (rows are 16-byte multiples)
    for (int i = threadIdx.x; i < H * (K1P / 8); i += blockDim.x) {
        const int r = i / (K1P / 8), c = i % (K1P / 8);
        *reinterpret_cast<uint4 *>(W1s + r * S1 + c * 8) = *reinterpret_cast<const uint4 *>(wt + G::w1 + (size_t)r * K1P + c * 8);
    }
    for (int i = threadIdx.x; i < H * (H / 8); i += blockDim.x) {
        const int r = i / (H / 8), c = i % (H / 8);
        *reinterpret_cast<uint4 *>(W2s + r * S2 + c * 8) = *reinterpret_cast<const uint4 *>(wt + G::w2 + (size_t)r * H + c * 8);
    }
    for (int i = threadIdx.x; i < 8 * (H / 8); i += blockDim.x) {
        const int r = i / (H / 8), c = i % (H / 8);
        *reinterpret_cast<uint4 *>(W3s + r * S2 + c * 8) = *reinterpret_cast<const uint4 *>(wt + G::w3 + (size_t)r * H + c * 8);
    }
    for (int i = threadIdx.x; i < 2 * H + 8; i += blockDim.x) Bs[i] = bias[i];
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const long long n_tiles = (n + 127) / 128;
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const long long r0 = tile * 128 + warp * 16 + g, r1 = r0 + 8;
        const float *x0 = x + r0 * NIN, *x1 = x + r1 * NIN;
        const bool v0 = r0 < n, v1 = r1 < n;
        // layer 1: acc = b1 + x W1
        float acc[NT][4];
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            acc[j][0] = acc[j][2] = Bs[8 * j + 2 * t];
            acc[j][1] = acc[j][3] = Bs[8 * j + 2 * t + 1];
        }
        float2 p[4], q[4];
        auto load = [&](int s, float2 (&f)[4]) {
            const int k0 = 16 * s + 2 * t, k1 = k0 + 8;
            const float2 z = make_float2(0.f, 0.f);
            f[0] = v0 && k0 < NIN ? *reinterpret_cast<const float2 *>(x0 + k0) : z;
            f[1] = v1 && k0 < NIN ? *reinterpret_cast<const float2 *>(x1 + k0) : z;
            f[2] = v0 && k1 < NIN ? *reinterpret_cast<const float2 *>(x0 + k1) : z;
            f[3] = v1 && k1 < NIN ? *reinterpret_cast<const float2 *>(x1 + k1) : z;
        };
        load(0, p);
#pragma unroll
        for (int s = 0; s < K1P / 16; ++s) {
            if (s + 1 < K1P / 16) load(s + 1, q);
            const uint32_t a[4] = {pack_bf16(p[0].x, p[0].y), pack_bf16(p[1].x, p[1].y), pack_bf16(p[2].x, p[2].y),
                                   pack_bf16(p[3].x, p[3].y)};
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const uint16_t *w = W1s + (8 * j + g) * S1 + 16 * s + 2 * t;
                mma_bf16(acc[j], a, *reinterpret_cast<const uint32_t *>(w), *reinterpret_cast<const uint32_t *>(w + 8));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) p[u] = q[u];
        }
        uint32_t af[NT / 2][4];
        to_frags<NT>(acc, af);
        // layer 2
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            acc[j][0] = acc[j][2] = Bs[H + 8 * j + 2 * t];
            acc[j][1] = acc[j][3] = Bs[H + 8 * j + 2 * t + 1];
        }
#pragma unroll
        for (int s = 0; s < G::KS; ++s)
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const uint16_t *w = W2s + (8 * j + g) * S2 + 16 * s + 2 * t;
                mma_bf16(acc[j], af[s], *reinterpret_cast<const uint32_t *>(w), *reinterpret_cast<const uint32_t *>(w + 8));
            }
        to_frags<NT>(acc, af);
        // layer 3 (6 outputs in one n-tile of 8)
        float o[4];
        o[0] = o[2] = Bs[2 * H + 2 * t];
        o[1] = o[3] = Bs[2 * H + 2 * t + 1];
#pragma unroll
        for (int s = 0; s < G::KS; ++s) {
            const uint16_t *w = W3s + g * S2 + 16 * s + 2 * t;
            mma_bf16(o, af[s], *reinterpret_cast<const uint32_t *>(w), *reinterpret_cast<const uint32_t *>(w + 8));
        }
        if (t < 3) {
            if (v0) *reinterpret_cast<float2 *>(out + r0 * NOUT + 2 * t) = make_float2(o[0], o[1]);
            if (v1) *reinterpret_cast<float2 *>(out + r1 * NOUT + 2 * t) = make_float2(o[2], o[3]);
        }
    }
}

template <int H>
int infer_h(tpx_ctx *c, const void *packed, const float *x, long long n, float *out) {
    using G = MlpGeo<H>;
    // the shared-memory attribute belongs to each device's context
    static std::atomic<bool> attr[64];
    int dev = 0, sms = 0;
    if (ck(cudaGetDevice(&dev)) || ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return TPX_ECUDA;
    const bool known = dev >= 0 && dev < 64;
    if (!known || !attr[dev].load(std::memory_order_acquire)) {
        if (ck(cudaFuncSetAttribute(k_mlp_bf16<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem)))
            return TPX_ECUDA;
        if (known) attr[dev].store(true, std::memory_order_release);
    }
    const long long tiles = (n + 127) / 128;
    const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);
    const uint16_t *wt = static_cast<const uint16_t *>(packed);
    const float *bias = reinterpret_cast<const float *>(static_cast<const char *>(packed) + packed_bias_off(G::wend));
    k_mlp_bf16<H><<<grid, 256, G::smem, c->stream>>>(x, n, wt, bias, out);
    return ck(cudaGetLastError()) ? TPX_ECUDA : TPX_OK;
}
template <int H>
int pack_h(tpx_ctx *c, const float *P, void *packed) {
    using G = MlpGeo<H>;
    uint16_t *wt = static_cast<uint16_t *>(packed);
    float *bias = reinterpret_cast<float *>(static_cast<char *>(packed) + packed_bias_off(G::wend));
    k_pack<H><<<grid_for((long long)G::wend + 2 * H + 8), 256, 0, c->stream>>>(P, wt, bias);
    return ck(cudaGetLastError()) ? TPX_ECUDA : TPX_OK;
}

}  // namespace tpxr

// the minibatch loss and its output gradient, and one Adam step, for the
// convolutional refiner (tpx_cnn.cu), which shares the loss and optimiser
int tpxr_loss(cudaStream_t s, const float *out, const float *y, int n, float w_off, float *dout, float *loss) {
    tpxr::k_loss<<<tpxr::grid_for(n), 256, 0, s>>>(out, y, n, w_off, dout, loss);
    return tpxr::ck(cudaGetLastError()) ? TPX_ECUDA : TPX_OK;
}
int tpxr_adam(cudaStream_t s, float *p, const float *g, float *m, float *v, long long n, float lr, long long step) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    tpxr::k_adam<<<tpxr::grid_for(n), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, c1, c2, 1e-8f);
    return tpxr::ck(cudaGetLastError()) ? TPX_ECUDA : TPX_OK;
}

using namespace tpxr;

template <typename OutT>
static int refine_patches(tpx_ctx *c, const uint64_t *d_packets, int64_t n, int64_t base, const int64_t *d_labels,
                          const tpx_record *d_clusters, int64_t n_clusters, int32_t min_pixels, OutT *d_patches,
                          int64_t *d_sel, int32_t *d_centre, int64_t capacity, int64_t *d_n_patches) {
    if (!c || n < 0 || n_clusters < 0 || capacity < 0 || !d_n_patches || min_pixels < 0) return TPX_EINVAL;
    if ((n > 0 && (!d_packets || !d_labels)) || (n_clusters > 0 && !d_clusters)) return TPX_EINVAL;
    if (capacity > 0 && (!d_patches || !d_sel || !d_centre)) return TPX_EINVAL;
    cudaStream_t s = c->stream;
    if (ck(cudaMemsetAsync(d_n_patches, 0, 8, s))) return TPX_ECUDA;
    if (n_clusters == 0 || n == 0) return TPX_OK;
    // scratch: flags, offsets, block sums, slot of each root packet, cell keys
    const long long nb = (n_clusters + SB - 1) / SB;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t need = 2 * al(4 * (size_t)n_clusters) + al(4 * (size_t)nb) + al(4 * (size_t)n) +
                        al(8 * (size_t)capacity * PC + 8);
    int rc = tpxg::reserve(c, need);
    if (rc) return rc;
    char *m = static_cast<char *>(c->g_mem);
    unsigned *f = reinterpret_cast<unsigned *>(m); m += al(4 * (size_t)n_clusters);
    unsigned *off = reinterpret_cast<unsigned *>(m); m += al(4 * (size_t)n_clusters);
    unsigned *bsum = reinterpret_cast<unsigned *>(m); m += al(4 * (size_t)nb);
    int *slot = reinterpret_cast<int *>(m); m += al(4 * (size_t)n);
    unsigned long long *key = reinterpret_cast<unsigned long long *>(m);
    k_sel_flags<<<grid_for(n_clusters), 256, 0, s>>>(d_clusters, n_clusters, min_pixels, f);
    k_scan_local<<<(unsigned)nb, SB, 0, s>>>(f, off, n_clusters, bsum);
    k_scan_sums<<<1, SB, 0, s>>>(bsum, nb, reinterpret_cast<long long *>(d_n_patches));
    k_scan_add<<<grid_for(n_clusters), 256, 0, s>>>(off, n_clusters, bsum);
    k_fill_i32<<<grid_for(n), 256, 0, s>>>(slot, n, -1);
    long long np = 0;
    if (ck(cudaMemcpyAsync(&np, d_n_patches, 8, cudaMemcpyDeviceToHost, s)) || ck(cudaStreamSynchronize(s)))
        return TPX_ECUDA;
    const long long ns = np < capacity ? np : capacity;
    k_select<<<grid_for(n_clusters), 256, 0, s>>>(d_packets, d_clusters, n_clusters, f, off, capacity, base, n,
                                                  reinterpret_cast<long long *>(d_sel), d_centre, slot);
    if (ns == 0) return ck(cudaGetLastError()) ? TPX_ECUDA : TPX_OK;
    if (ck(cudaMemsetAsync(key, 0, 8 * (size_t)ns * PC, s))) return TPX_ECUDA;
    k_patch_keys<<<grid_for(n), 256, 0, s>>>(d_packets, n, base, reinterpret_cast<const long long *>(d_labels), slot,
                                             d_centre, key);
    k_patch_fill<OutT><<<grid_for(ns * PC), 256, 0, s>>>(d_packets, base, d_clusters,
                                                         reinterpret_cast<const long long *>(d_sel), key, ns, d_patches);
    if (ck(cudaGetLastError())) return TPX_ECUDA;
    return np > capacity ? TPX_EOVERFLOW : TPX_OK;
}

extern "C" {

int tpx_refine_patches(tpx_ctx *c, const uint64_t *d_packets, int64_t n, int64_t base, const int64_t *d_labels,
                       const tpx_record *d_clusters, int64_t n_clusters, int32_t min_pixels, float *d_patches,
                       int64_t *d_sel, int32_t *d_centre, int64_t capacity, int64_t *d_n_patches) {
    return refine_patches<float>(c, d_packets, n, base, d_labels, d_clusters, n_clusters, min_pixels, d_patches, d_sel,
                                 d_centre, capacity, d_n_patches);
}

int tpx_refine_patches_bf16(tpx_ctx *c, const uint64_t *d_packets, int64_t n, int64_t base, const int64_t *d_labels,
                            const tpx_record *d_clusters, int64_t n_clusters, int32_t min_pixels, uint16_t *d_patches,
                            int64_t *d_sel, int32_t *d_centre, int64_t capacity, int64_t *d_n_patches) {
    return refine_patches<uint16_t>(c, d_packets, n, base, d_labels, d_clusters, n_clusters, min_pixels, d_patches,
                                    d_sel, d_centre, capacity, d_n_patches);
}

int64_t tpx_refiner_params(int32_t hidden) { return hidden > 0 ? Layout(hidden).total : 0; }

// forward pass; `act` (n x (2H + NOUT) floats) keeps the activations for a
// backward pass, or may be NULL when `out` is given
static int forward(tpx_ctx *c, const float *P, int h, const float *x, int64_t n, float *a1, float *a2, float *out) {
    const Layout L(h);
    cudaStream_t s = c->stream;
    // rows in chunks the GEMM grid can hold (grid.y <= 65535 tiles of 64 rows)
    constexpr int64_t kRows = 1LL << 21;
    for (int64_t r0 = 0; r0 < n; r0 += kRows) {
        const int m = (int)(n - r0 < kRows ? n - r0 : kRows);
        gemm(s, x + r0 * NIN, NIN, 1, P + L.w1, h, 1, a1 + r0 * h, h, m, h, NIN, P + L.b1, true);
        gemm(s, a1 + r0 * h, h, 1, P + L.w2, h, 1, a2 + r0 * h, h, m, h, h, P + L.b2, true);
        gemm(s, a2 + r0 * h, h, 1, P + L.w3, NOUT, 1, out + r0 * NOUT, NOUT, m, NOUT, h, P + L.b3, false);
    }
    return ck(cudaGetLastError()) ? TPX_ECUDA : TPX_OK;
}

int tpx_refiner_forward(tpx_ctx *c, const float *d_params, int32_t hidden, const float *d_x, int64_t n,
                        float *d_work, float *d_out) {
    if (!c || !d_params || hidden < 1 || n < 0 || (n > 0 && (!d_x || !d_work || !d_out)) || n >= (1LL << 31))
        return TPX_EINVAL;
    if (n == 0) return TPX_OK;
    return forward(c, d_params, hidden, d_x, n, d_work, d_work + (long long)n * hidden, d_out);
}

int tpx_refiner_train_step(tpx_ctx *c, float *d_params, float *d_adam_m, float *d_adam_v, float *d_grad,
                           int32_t hidden, int64_t step, const float *d_x, const float *d_y, int64_t n, float lr,
                           float offset_weight, float *d_work, float *d_loss) {
    if (!c || !d_params || !d_adam_m || !d_adam_v || !d_grad || hidden < 1 || step < 1 || !d_x || !d_y || n < 1 ||
        !d_work || !d_loss || n > (1LL << 21))
        return TPX_EINVAL;
    const Layout L(hidden);
    const int h = hidden;
    cudaStream_t s = c->stream;
    float *a1 = d_work, *a2 = a1 + (long long)n * h, *out = a2 + (long long)n * h;
    float *dout = out + (long long)n * NOUT, *d2 = dout + (long long)n * NOUT, *d1 = d2 + (long long)n * h;
    int rc = forward(c, d_params, h, d_x, n, a1, a2, out);
    if (rc) return rc;
    if (ck(cudaMemsetAsync(d_loss, 0, 4, s))) return TPX_ECUDA;
    k_loss<<<grid_for(n), 256, 0, s>>>(out, d_y, (int)n, offset_weight, dout, d_loss);
    // layer 3: dW3 = a2^T dout, db3 = colsum(dout), d2 = dout W3^T
    gemm(s, a2, 1, h, dout, NOUT, 1, d_grad + L.w3, NOUT, h, NOUT, (int)n, nullptr, false);
    k_colsum<<<1, 256, 0, s>>>(dout, (int)n, NOUT, d_grad + L.b3);
    gemm(s, dout, NOUT, 1, d_params + L.w3, 1, NOUT, d2, h, (int)n, h, NOUT, nullptr, false);
    k_relu_back<<<grid_for((long long)n * h), 256, 0, s>>>(d2, a2, (long long)n * h);
    // layer 2
    gemm(s, a1, 1, h, d2, h, 1, d_grad + L.w2, h, h, h, (int)n, nullptr, false);
    k_colsum<<<(h + 255) / 256, 256, 0, s>>>(d2, (int)n, h, d_grad + L.b2);
    gemm(s, d2, h, 1, d_params + L.w2, 1, h, d1, h, (int)n, h, h, nullptr, false);
    k_relu_back<<<grid_for((long long)n * h), 256, 0, s>>>(d1, a1, (long long)n * h);
    // layer 1
    gemm(s, d_x, 1, NIN, d1, h, 1, d_grad + L.w1, h, NIN, h, (int)n, nullptr, false);
    k_colsum<<<(h + 255) / 256, 256, 0, s>>>(d1, (int)n, h, d_grad + L.b1);
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<grid_for(L.total), 256, 0, s>>>(d_params, d_grad, d_adam_m, d_adam_v, L.total, lr, b1, b2, c1, c2, 1e-8f);
    return ck(cudaGetLastError()) ? TPX_ECUDA : TPX_OK;
}

int64_t tpx_refiner_packed_bytes(int32_t hidden) {
    switch (hidden) {
        case 64: return (int64_t)MlpGeo<64>::packed_bytes;
        case 128: return (int64_t)MlpGeo<128>::packed_bytes;
        case 160: return (int64_t)MlpGeo<160>::packed_bytes;
        default: return 0;
    }
}

int tpx_refiner_pack(tpx_ctx *c, const float *d_params, int32_t hidden, void *d_packed) {
    if (!c || !d_params || !d_packed || (reinterpret_cast<uintptr_t>(d_packed) & 15)) return TPX_EINVAL;
    switch (hidden) {
        case 64: return pack_h<64>(c, d_params, d_packed);
        case 128: return pack_h<128>(c, d_params, d_packed);
        case 160: return pack_h<160>(c, d_params, d_packed);
        default: return TPX_EUNSUPPORTED;
    }
}

int tpx_refiner_infer(tpx_ctx *c, const void *d_packed, int32_t hidden, const float *d_x, int64_t n, float *d_out) {
    if (!c || n < 0 || (n > 0 && (!d_packed || !d_x || !d_out))) return TPX_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_packed) & 15) || (reinterpret_cast<uintptr_t>(d_x) & 7) ||
        (reinterpret_cast<uintptr_t>(d_out) & 7))
        return TPX_EINVAL;
    if (hidden != 64 && hidden != 128 && hidden != 160) return TPX_EUNSUPPORTED;
    if (n == 0) return TPX_OK;
    switch (hidden) {
        case 64: return infer_h<64>(c, d_packed, d_x, n, d_out);
        case 128: return infer_h<128>(c, d_packed, d_x, n, d_out);
        default: return infer_h<160>(c, d_packed, d_x, n, d_out);
    }
}

int tpx_refine_decide(tpx_ctx *c, const float *d_out, const tpx_record *d_clusters, const int64_t *d_sel,
                      const int32_t *d_centre, int64_t n, float threshold, float *d_hits) {
    if (!c || n < 0 || (n > 0 && (!d_out || !d_clusters || !d_sel || !d_centre || !d_hits))) return TPX_EINVAL;
    if (!(threshold > 0.f && threshold < 1.f)) return TPX_EINVAL;
    if (n == 0) return TPX_OK;
    const float lt = (float)std::log((double)threshold / (1.0 - (double)threshold));
    k_decide<<<grid_for(n), 256, 0, c->stream>>>(d_out, d_clusters, reinterpret_cast<const long long *>(d_sel),
                                                 d_centre, n, lt, d_hits);
    return ck(cudaGetLastError()) ? TPX_ECUDA : TPX_OK;
}

}  // extern "C"
