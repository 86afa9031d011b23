// tpx_cnn.cu -- the convolutional overlap refiner (not in the paper; its
// multi-hit discussion, Sec. VII.B, and the local-maximum count of Sec. V.B
// motivate it): the 9 x 9 patch of a cluster (channel 0: ToT, channel 1:
// relative ToA) through three 3 x 3 convolutions without padding and two
// dense layers, to one or two particles and their sub-pixel offsets.
//
//   conv1  2 -> 16 channels, 9 x 9 -> 7 x 7, ReLU
//   conv2 16 -> 16 channels, 7 x 7 -> 5 x 5, ReLU
//   conv3 16 -> 32 channels, 5 x 5 -> 3 x 3, ReLU
//   fc1   288 -> 144, ReLU (a 3 x 3 convolution of the 3 x 3 map to 1 x 1)
//   fc2   144 -> 6 (two count logits, (dx, dy) of each particle)
// 49,750 parameters, one fp32 array: W1 [16][2][3][3], b1, W2 [16][16][3][3],
// b2, W3 [32][16][3][3], b3, W4 [144][288] (inputs in channel, row, column
// order), b4, W5 [6][144], b5.
//
// Training (fp32): every layer is a GEMM of the layer's im2col matrix (rows:
// output positions of all patches; columns: input channel, kernel row,
// kernel column) with the weights; the backward pass uses the same matrices
// (weight gradients as split-K GEMMs over the rows, input gradients gathered
// back from the column gradients). Inference: one kernel runs all five layers
// on the fifth-generation tensor cores for groups of patches -- implicit GEMMs
// whose A operands are the layers' input maps in shared memory, read through
// shifted descriptors (no im2col copy); one thread issues tcgen05.mma (bf16
// operands, fp32 accumulators in tensor memory), the epilogue reads the
// accumulators with tcgen05.ld, adds the bias, applies the ReLU and rounds
// the activation to bf16 into the next layer's input map.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "tpx.h"
#include "tpx_ctx.h"
#include "tpx_fused.cuh"

namespace tpxc {

constexpr int NOUT = 6;
constexpr int NPARAM = 49750;

// parameter offsets (floats)
constexpr long long OW1 = 0, OB1 = OW1 + 16 * 2 * 9, OW2 = OB1 + 16, OB2 = OW2 + 16 * 16 * 9, OW3 = OB2 + 16,
                    OB3 = OW3 + 32 * 16 * 9, OW4 = OB3 + 32, OB4 = OW4 + 144 * 288, OW5 = OB4 + 144,
                    OB5 = OW5 + NOUT * 144, OEND = OB5 + NOUT;
static_assert(OEND == NPARAM, "parameter count");

inline bool ck(cudaError_t e, int line = __builtin_LINE()) {
    if (e == cudaSuccess) return false;
    if (std::getenv("TPX_DEBUG")) std::fprintf(stderr, "tpx_cnn.cu:%d: %s\n", line, cudaGetErrorString(e));
    return true;
}
inline unsigned grid_for(long long n, int bt = 256) {
    long long g = (n + bt - 1) / bt;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)g;
}

// one convolution layer (3 x 3, or the 1 x 1 of fc2): input hin x hin x cin,
// output ho x ho x cout
struct Conv { int cin, hin, cout, ho, kk; long long ow, ob; };   // kk: kernel side (3 or 1)
__host__ __device__ constexpr Conv layer_of(int l) {
    return l == 0 ? Conv{2, 9, 16, 7, 3, OW1, OB1} : l == 1 ? Conv{16, 7, 16, 5, 3, OW2, OB2}
         : l == 2 ? Conv{16, 5, 32, 3, 3, OW3, OB3} : l == 3 ? Conv{32, 3, 144, 1, 3, OW4, OB4}
                  : Conv{144, 1, NOUT, 1, 1, OW5, OB5};
}

// ================================================================ fp32 training
// im2col: out[(p, oy, ox)][ci * kk^2 + ky * kk + kx] = in(p, oy + ky, ox + kx, ci)
// with in(p, y, x, c) = in[p * sn + y * sy + x * sx + c * sc]
__global__ void k_im2col(const float *in, long long sn, int sy, int sx, int sc, long long n, int cin, int ho, int kk,
                         float *out) {
    const int K = cin * kk * kk;
    const long long total = n * ho * ho * K;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % K);
        const long long r = i / K;
        const int ox = (int)(r % ho), oy = (int)((r / ho) % ho);
        const long long p = r / ((long long)ho * ho);
        const int ci = k / (kk * kk), t = k % (kk * kk), ky = t / kk, kx = t % kk;
        out[i] = in[p * sn + (long long)(oy + ky) * sy + (long long)(ox + kx) * sx + (long long)ci * sc];
    }
}
// the input gradient from the im2col gradient: each input element gathers the
// columns that read it; out rows (p, y, x) x cin
__global__ void k_col2im(const float *dcol, long long n, int cin, int hin, int ho, int kk, float *out) {
    const int K = cin * kk * kk;
    const long long total = n * hin * hin * cin;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % cin);
        const long long r = i / cin;
        const int x = (int)(r % hin), y = (int)((r / hin) % hin);
        const long long p = r / ((long long)hin * hin);
        float s = 0.f;
        for (int ky = 0; ky < kk; ++ky) {
            const int oy = y - ky;
            if (oy < 0 || oy >= ho) continue;
            for (int kx = 0; kx < kk; ++kx) {
                const int ox = x - kx;
                if (ox < 0 || ox >= ho) continue;
                s += dcol[((p * ho + oy) * ho + ox) * K + ci * kk * kk + ky * kk + kx];
            }
        }
        out[i] = s;
    }
}

// C[M x N] (+)= op(A)[M x K] op(B)[K x N] (+ bias, ReLU), strides as in the
// MLP refiner's GEMM; gridDim.z > 1 splits K and adds the partial products
// atomically into C (zeroed by the caller; no bias or ReLU then)
constexpr int TM = 64, TN = 64, TK = 16;
__global__ void __launch_bounds__(256) k_sgemm(const float *A, long long sam, long long sak, const float *B,
                                               long long sbk, long long sbn, float *C, long long ldc, int M, int N,
                                               long long K, const float *bias, int relu) {
    __shared__ float As[TK][TM + 4];
    __shared__ float Bs[TK][TN + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
    const long long kc = (K + gridDim.z - 1) / gridDim.z;
    const long long kb = blockIdx.z * kc, ke = min(K, kb + kc);
    float acc[4][4] = {};
    for (long long k0 = kb; k0 < ke; k0 += TK) {
        for (int t = threadIdx.x; t < TK * TM; t += 256) {
            const int kk = sak == 1 ? t % TK : t / TM, ii = sak == 1 ? t / TK : t % TM;
            const int i = i0 + ii;
            const long long k = k0 + kk;
            As[kk][ii] = (i < M && k < ke) ? A[i * sam + k * sak] : 0.f;
        }
        for (int t = threadIdx.x; t < TK * TN; t += 256) {
            const int kk = sbk == 1 ? t % TK : t / TN, jj = sbk == 1 ? t / TK : t % TN;
            const int j = j0 + jj;
            const long long k = k0 + kk;
            Bs[kk][jj] = (j < N && k < ke) ? B[k * sbk + j * sbn] : 0.f;
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
            float *c = C + (long long)i * ldc + j;
            if (gridDim.z > 1) { atomicAdd(c, acc[r][q]); continue; }
            float v = acc[r][q];
            if (bias) v += bias[j];
            if (relu) v = fmaxf(v, 0.f);
            *c = v;
        }
}
void sgemm(cudaStream_t s, const float *A, long long sam, long long sak, const float *B, long long sbk, long long sbn,
           float *C, long long ldc, long long M, int N, long long K, const float *bias, bool relu, int splits = 1) {
    constexpr long long kRows = 1LL << 21;   // grid.y <= 65535 tiles of 64 rows
    for (long long m0 = 0; m0 < M; m0 += kRows) {
        const int m = (int)(M - m0 < kRows ? M - m0 : kRows);
        dim3 g((N + TN - 1) / TN, (m + TM - 1) / TM, splits);
        k_sgemm<<<g, 256, 0, s>>>(A + m0 * sam, sam, sak, B, sbk, sbn, C + m0 * ldc, ldc, m, N, K, bias, relu ? 1 : 0);
    }
}
// splits for a weight gradient whose inner dimension runs over `rows`
inline int splits_for(long long rows, int M, int N) {
    const long long tiles = (long long)((M + TM - 1) / TM) * ((N + TN - 1) / TN);
    long long sp = (152LL * 4) / (tiles > 0 ? tiles : 1);
    const long long per = rows / 1024;   // at least ~1024 rows per split
    if (sp > per) sp = per;
    return (int)(sp < 1 ? 1 : (sp > 65535 ? 65535 : sp));
}

__global__ void k_relu_back(float *d, const float *act, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (act[i] <= 0.f) d[i] = 0.f;
}
// column sums of d [rows x m] added into g (m <= blockDim.x): per block a
// strip of rows, blockDim.x / m row lanes per column
__global__ void k_colsum(const float *d, long long rows, int m, float *g) {
    const int lanes = blockDim.x / m;
    const int j = threadIdx.x % m, rl = threadIdx.x / m;
    if (rl >= lanes) return;
    const long long per = (rows + gridDim.x - 1) / gridDim.x;
    const long long r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
    float s = 0.f;
    for (long long r = r0 + rl; r < r1; r += lanes) s += d[r * m + j];
    atomicAdd(&g[j], s);
}

// rows, workspace floats per patch
constexpr long long kWork = 49 * 18 + 49 * 16 + 25 * 144 + 25 * 16 + 9 * 144 + 9 * 32 + 288 + 144 + 2 * NOUT +
                            144 + 288 + 9 * 32 + 9 * 144 + 25 * 16 + 25 * 144 + 49 * 16;

struct Work {
    float *x1, *a1, *x2, *a2, *x3, *a3, *x4, *a4, *out, *dout, *d4, *dx4, *d3, *dx3, *d2, *dx2, *d1;
    Work(float *w, long long n) {
        float *p = w;
        auto take = [&](long long per) { float *r = p; p += per * n; return r; };
        x1 = take(49 * 18); a1 = take(49 * 16); x2 = take(25 * 144); a2 = take(25 * 16); x3 = take(9 * 144);
        a3 = take(9 * 32); x4 = take(288); a4 = take(144); out = take(NOUT); dout = take(NOUT); d4 = take(144);
        dx4 = take(288); d3 = take(9 * 32); dx3 = take(9 * 144); d2 = take(25 * 16); dx2 = take(25 * 144);
        d1 = take(49 * 16);
    }
};

// the fp32 forward pass of n patches (x: [n][162], channel 0 then 1, rows of 9)
int forward32(cudaStream_t s, const float *P, const float *x, long long n, const Work &w) {
    k_im2col<<<grid_for(n * 49 * 18), 256, 0, s>>>(x, 162, 9, 1, 81, n, 2, 7, 3, w.x1);
    sgemm(s, w.x1, 18, 1, P + OW1, 1, 18, w.a1, 16, n * 49, 16, 18, P + OB1, true);
    k_im2col<<<grid_for(n * 25 * 144), 256, 0, s>>>(w.a1, 49 * 16, 7 * 16, 16, 1, n, 16, 5, 3, w.x2);
    sgemm(s, w.x2, 144, 1, P + OW2, 1, 144, w.a2, 16, n * 25, 16, 144, P + OB2, true);
    k_im2col<<<grid_for(n * 9 * 144), 256, 0, s>>>(w.a2, 25 * 16, 5 * 16, 16, 1, n, 16, 3, 3, w.x3);
    sgemm(s, w.x3, 144, 1, P + OW3, 1, 144, w.a3, 32, n * 9, 32, 144, P + OB3, true);
    k_im2col<<<grid_for(n * 288), 256, 0, s>>>(w.a3, 9 * 32, 3 * 32, 32, 1, n, 32, 1, 3, w.x4);
    sgemm(s, w.x4, 288, 1, P + OW4, 1, 288, w.a4, 144, n, 144, 288, P + OB4, true);
    sgemm(s, w.a4, 144, 1, P + OW5, 1, 144, w.out, NOUT, n, NOUT, 144, P + OB5, false);
    return ck(cudaGetLastError()) ? TPX_ECUDA : TPX_OK;
}

// weight and bias gradients of one layer from dZ [rows x cout] and its
// im2col matrix X [rows x K]; dX = dZ W [rows x K] when wanted
void layer_back(cudaStream_t s, const float *P, float *G, const Conv &L, const float *X, const float *dZ, long long rows,
                float *dX) {
    const int K = L.cin * L.kk * L.kk;
    sgemm(s, dZ, 1, L.cout, X, K, 1, G + L.ow, K, L.cout, K, rows, nullptr, false, splits_for(rows, L.cout, K));
    k_colsum<<<grid_for(rows / 64 + 1), 256, 0, s>>>(dZ, rows, L.cout, G + L.ob);
    if (dX) sgemm(s, dZ, L.cout, 1, P + L.ow, K, 1, dX, K, rows, K, L.cout, nullptr, false);
}

// ================================================================ inference
// tcgen05 implicit GEMM per layer. Shared-memory operands use the canonical
// K-major layout without swizzle: 8 x 16-byte core matrices (8 rows, 8 bf16
// along K), core (i, j) -- row group i, k group j -- at (i * K / 8 + j) * 128
// bytes; a descriptor's leading offset (between core matrices along K) is 128
// bytes, its stride offset (between row groups) K / 8 * 128 bytes.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);   // version 1, no swizzle
}
// instruction descriptor: dense kind::f16, bf16 A and B (K-major), fp32 D, M = 128
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// byte offset of element (r, k) of a core-matrix tile with KP columns
__device__ __forceinline__ uint32_t core_off(int r, int k, int kp) {
    return (uint32_t)((((r >> 3) * (kp >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

constexpr long long kSpin = 1LL << 24;   // bounded mbarrier wait (then an error flag)

// asynchronous global -> shared copies (16 or 4 bytes; 0 source bytes fill zeros)
__device__ __forceinline__ void cp16(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// packed inference weights: per layer [N][KP] bf16 with column k = tap * cin +
// ci (8 channels of a tap per 16-byte chunk; conv1: ky * 8 + kx * 2 + ci, one
// chunk per kernel row), zero padded; then the biases (fp32, padded to N)
struct Packed {
    static constexpr int N1 = 16, KP1 = 32, N2 = 16, KP2 = 144, N3 = 32, KP3 = 144, N4 = 144, KP4 = 288, N5 = 16,
                         KP5 = 144;
    static constexpr size_t w1 = 0, w2 = w1 + (size_t)N1 * KP1, w3 = w2 + (size_t)N2 * KP2, w4 = w3 + (size_t)N3 * KP3,
                            w5 = w4 + (size_t)N4 * KP4, wend = w5 + (size_t)N5 * KP5;
    static constexpr size_t boff = ((wend * 2 + 255) / 256) * 256;   // bytes
    static constexpr size_t b1 = 0, b2 = b1 + N1, b3 = b2 + N2, b4 = b3 + N3, b5 = b4 + N4, bend = b5 + N5;
    static constexpr size_t bytes = boff + bend * 4;
};

__global__ void k_cnn_pack(const float *P, __nv_bfloat16 *wt, float *bias) {
    using Q = Packed;
    const long long total = (long long)Q::wend + (long long)Q::bend;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        if (i >= (long long)Q::wend) {
            const int b = (int)(i - Q::wend);
            float v = 0.f;
            if (b < (int)Q::b2) v = P[OB1 + b];
            else if (b < (int)Q::b3) v = P[OB2 + b - Q::b2];
            else if (b < (int)Q::b4) v = P[OB3 + b - Q::b3];
            else if (b < (int)Q::b5) v = P[OB4 + b - Q::b4];
            else if (b - (int)Q::b5 < NOUT) v = P[OB5 + b - Q::b5];
            bias[b] = v;
            continue;
        }
        float v = 0.f;
        int L, r, k;
        long long o;
        if (i < (long long)Q::w2) { L = 0; o = i - Q::w1; r = (int)(o / Q::KP1); k = (int)(o % Q::KP1); }
        else if (i < (long long)Q::w3) { L = 1; o = i - Q::w2; r = (int)(o / Q::KP2); k = (int)(o % Q::KP2); }
        else if (i < (long long)Q::w4) { L = 2; o = i - Q::w3; r = (int)(o / Q::KP3); k = (int)(o % Q::KP3); }
        else if (i < (long long)Q::w5) { L = 3; o = i - Q::w4; r = (int)(o / Q::KP4); k = (int)(o % Q::KP4); }
        else { L = 4; o = i - Q::w5; r = (int)(o / Q::KP5); k = (int)(o % Q::KP5); }
        const Conv C = layer_of(L);
        const int kk2 = C.kk * C.kk, K = C.cin * kk2;
        if (L == 0) {   // conv1: one 8-wide chunk per kernel row, [c0, c1] at kx = 0, 1, 2, two zeros
            const int ky = k / 8, kx = (k % 8) / 2, ci = k % 2;
            if (r < C.cout && ky < 3 && k % 8 < 6) v = P[C.ow + (long long)r * K + ci * kk2 + ky * 3 + kx];
        } else if (r < C.cout && k < K) {   // k = tap * cin + ci: 8 channels of a tap per chunk
            const int t = k / C.cin, ci = k % C.cin;
            v = P[C.ow + (long long)r * K + ci * kk2 + t];   // [cout][cin][tap]
        }
        wt[i] = __float2bfloat16_rn(v);
    }
}

// ---------------------------------------------------------------- fused inference
// One persistent CTA per SM carries groups of FP patches through all five
// layers: the activations stay in one shared-memory region X (each layer's
// input is dead once its MMAs completed, so the next layer's input takes its
// place), the accumulators in tensor memory, the weights in shared memory for
// the whole launch. The convolutions are implicit GEMMs with no im2col copy:
// a layer's input map is stored as planes of 8 channels with one 16-byte row
// per input position, and the layer computes an output row for every position
// of its input grid (the rows outside the valid window are computed and
// dropped), so the A operand of kernel tap (ky, kx) is the map itself shifted
// by ky * W + kx rows -- a descriptor with its start moved, leading offset the
// plane stride, stride offset one core matrix (8 rows). conv1's two channels
// are packed with those of the two right-hand neighbours into one row
// ([c0, c1] at x, x + 1, x + 2, then two zeros), so a k chunk is a kernel row.
// Rows past the valid ones read stale (finite) contents of X; X starts zeroed.
constexpr int FP = 48;                                // patches per group
constexpr int R1 = FP * 81, T1 = (R1 + 127) / 128;    // conv1: rows of the 9 x 9 grid, MMA tiles
constexpr int R2 = FP * 49, T2 = (R2 + 127) / 128;    // conv2: 7 x 7 grid
constexpr int R3 = FP * 25, T3 = (R3 + 127) / 128;    // conv3: 5 x 5 grid
constexpr int M1_ROWS = T1 * 128 + 27;                // conv1 reads up to the largest shift (18, then +9)
constexpr int P1_ROWS = T2 * 128 + 16;                // conv2 input plane (shifts up to 2 * 7 + 2)
constexpr int P2_ROWS = T3 * 128 + 12;                // conv3 input plane (shifts up to 2 * 5 + 2)
constexpr int PLB = FP * 16;                          // dense-layer input plane: one row per patch
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t X_BYTES =
    ((cmax(cmax((size_t)M1_ROWS * 16, (size_t)2 * P1_ROWS * 16),
           cmax((size_t)2 * P2_ROWS * 16, cmax((size_t)(35 * FP + 128) * 16, (size_t)(17 * FP + 128) * 16))) +
      127) / 128) * 128;
constexpr size_t W1B = 16 * 32 * 2, W2B = 16 * 144 * 2, W3B = 32 * 144 * 2, W4B = 144 * 288 * 2, W5B = 16 * 144 * 2;
constexpr size_t W_BYTES = W1B + W2B + W3B + W4B + W5B;
constexpr size_t RAW_BYTES = (size_t)FP * 162 * 2;    // one group of bf16 patches
constexpr size_t BIAS_BYTES = ((Packed::bend * 4 + 127) / 128) * 128;
constexpr size_t FUSED_SMEM = 1024 + W_BYTES + X_BYTES + 2 * RAW_BYTES + BIAS_BYTES + 64;
static_assert(T1 * 16 <= 512 && T2 * 16 <= 512 && T3 * 32 <= 512 && FP <= 128, "tensor memory of a group");
static_assert(FUSED_SMEM <= 227 * 1024, "shared memory of the fused kernel");
static_assert(RAW_BYTES % 16 == 0 && W_BYTES % 128 == 0, "16-byte copies");

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, bool acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc ? 1u : 0u)
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t ta, uint32_t *v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// 32 consecutive accumulator columns of the warp's 32 lanes, no wait
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t ta, uint32_t *v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(ta));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 16 accumulators + bias, ReLU, rounded to bf16: two 16-byte rows of 8 channels
__device__ __forceinline__ void relu_bf16x16(const uint32_t *v, const float *bias, uint4 *lo, uint4 *hi) {
    uint32_t pk[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float a = fmaxf(__uint_as_float(v[2 * j]) + bias[2 * j], 0.f);
        const float b = fmaxf(__uint_as_float(v[2 * j + 1]) + bias[2 * j + 1], 0.f);
        __nv_bfloat162 b2 = __floats2bfloat162_rn(a, b);
        pk[j] = *reinterpret_cast<uint32_t *>(&b2);
    }
    *lo = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    *hi = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

// [N][KP] bf16 rows of the packed weights into the canonical core-matrix layout
__device__ __forceinline__ void load_weights(unsigned char *dst, const __nv_bfloat16 *w, int n, int kp) {
    for (int i = threadIdx.x; i < n * (kp / 8); i += blockDim.x) {
        const int r = i / (kp / 8), c = i % (kp / 8);
        *reinterpret_cast<uint4 *>(dst + core_off(r, c * 8, kp)) = *reinterpret_cast<const uint4 *>(w + (size_t)r * kp + c * 8);
    }
}

// the bf16 patches of group g (zero past the last patch), 16-byte copies
__device__ __forceinline__ void load_group(unsigned char *raw, const __nv_bfloat16 *x, long long n, long long g) {
    const long long b0 = g * (long long)RAW_BYTES, bend = n * 324;
    const unsigned char *src = reinterpret_cast<const unsigned char *>(x);
    for (int i = threadIdx.x; i < (int)(RAW_BYTES / 16); i += blockDim.x) {
        const long long o = b0 + 16LL * i;
        const long long rem = bend - o;
        const int bytes = rem >= 16 ? 16 : (rem > 0 ? (int)rem : 0);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(raw + 16 * i)),
                     "l"(src + (bytes ? o : 0)), "r"(bytes)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

constexpr int CNN_THREADS = 512;   // 16 warps: four per tensor-memory lane quadrant

// Phase timing (-DTPX_PHASE_TIMING, the libtpx_phases.so build): thread 0 of
// every CTA adds the clock64 cycles since its previous mark to the phase's
// counter (read with tpx_debug_cnn_phase_times); compiled away otherwise.
#ifdef TPX_PHASE_TIMING
__device__ unsigned long long g_cnn_phase[16];
#define CNN_PH(k)                                                                                       \
    do {                                                                                                \
        const long long ph_now = clock64();                                                             \
        if (threadIdx.x == 0) atomicAdd(&g_cnn_phase[k], (unsigned long long)(ph_now - ph_t));           \
        ph_t = ph_now;                                                                                  \
    } while (0)
#else
#define CNN_PH(k) do {} while (0)
#endif

__global__ void __launch_bounds__(CNN_THREADS, 1) k_cnn_fused(const __nv_bfloat16 *__restrict__ x, long long n,
                                                      const __nv_bfloat16 *__restrict__ wt,
                                                      const float *__restrict__ bias, float *__restrict__ out,
                                                      unsigned *status) {
    using Q = Packed;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *W1 = base, *W2 = W1 + W1B, *W3 = W2 + W2B, *W4 = W3 + W3B, *W5 = W4 + W4B;
    unsigned char *X = W5 + W5B;
    unsigned char *RAW[2] = {X + X_BYTES, X + X_BYTES + RAW_BYTES};
    float *SB = reinterpret_cast<float *>(X + X_BYTES + 2 * RAW_BYTES);   // the biases
    uint64_t *bar = reinterpret_cast<uint64_t *>(X + X_BYTES + 2 * RAW_BYTES + BIAS_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, sub = warp >> 2;   // accumulator lanes 32 * quad.., and which share of the columns
    const long long groups = (n + FP - 1) / FP;

    load_weights(W1, wt + Q::w1, 16, 32);
    load_weights(W2, wt + Q::w2, 16, 144);
    load_weights(W3, wt + Q::w3, 32, 144);
    load_weights(W4, wt + Q::w4, 144, 288);
    load_weights(W5, wt + Q::w5, 16, 144);
    for (int i = tid; i < (int)(X_BYTES / 16); i += CNN_THREADS) reinterpret_cast<uint4 *>(X)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < (int)Q::bend; i += CNN_THREADS) SB[i] = bias[i];
    if (tid == 0) mbar_init(smem_u32(bar), 4);   // four issuing threads commit per layer
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    long long g = blockIdx.x;
    if (g < groups) load_group(RAW[0], x, n, g);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t xs = smem_u32(X);
    const uint32_t lane_off = (uint32_t)(32 * quad) << 16;   // this warp's accumulator lanes
    uint32_t phase = 0;
    bool failed = false;
#ifdef TPX_PHASE_TIMING
    long long ph_t = clock64();
#endif

    // the layer's A operand is in X: make it visible to the tensor cores, then
    // lane 0 of warps 0-3 (one per scheduler) each issue a share of the MMAs
    // and commit them to the barrier (four arrivals); everyone waits (bounded)
    const int issuer = (lane == 0 && warp < 4) ? warp : -1;
    auto run_layer = [&](auto issue) -> bool {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (issuer >= 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            issue(issuer);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                         : "memory");
        }
        long long spins = 0;
        bool bad = false;
        while (!mbar_try_wait(smem_u32(bar), phase)) {
            if (++spins > kSpin) { bad = true; break; }
        }
        phase ^= 1u;
        if (__syncthreads_or(bad ? 1 : 0)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return true;
    };

    for (int it = 0; g < groups; g += gridDim.x, ++it) {
        unsigned char *raw = RAW[it & 1];
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        CNN_PH(0);
        // the next group's patches come in while this one runs
        if (g + gridDim.x < groups) load_group(RAW[(it + 1) & 1], x, n, g + gridDim.x);
        // ---- conv1 input map: row (patch, y * 9 + x) = [c0, c1] at x, x + 1, x + 2, 0, 0 ----
        {
            const __nv_bfloat16 *pr = reinterpret_cast<const __nv_bfloat16 *>(raw);
            for (int r = tid; r < R1; r += CNN_THREADS) {
                const int pp = r / 81, pos = r % 81, xx = pos % 9;
                const __nv_bfloat16 *c0 = pr + pp * 162 + pos, *c1 = c0 + 81;
                const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
                __nv_bfloat162 v0 = __halves2bfloat162(c0[0], c1[0]);
                __nv_bfloat162 v1 = xx + 1 < 9 ? __halves2bfloat162(c0[1], c1[1]) : __halves2bfloat162(z, z);
                __nv_bfloat162 v2 = xx + 2 < 9 ? __halves2bfloat162(c0[2], c1[2]) : __halves2bfloat162(z, z);
                __nv_bfloat162 v3 = __halves2bfloat162(z, z);
                uint4 row;
                row.x = *reinterpret_cast<uint32_t *>(&v0);
                row.y = *reinterpret_cast<uint32_t *>(&v1);
                row.z = *reinterpret_cast<uint32_t *>(&v2);
                row.w = *reinterpret_cast<uint32_t *>(&v3);
                reinterpret_cast<uint4 *>(X)[r] = row;
            }
        }
        CNN_PH(1);
        // ---- conv1: 2 MMAs per tile (kernel rows 0-1, then row 2 and a zero chunk) ----
        if (!run_layer([&](int q) {
                // a descriptor's start field counts 16-byte units: one row, or
                // 256 bytes = 16 for the next two k chunks of the weights
                const uint32_t id = idesc_bf16(16);
                const uint64_t da = sdesc(xs, 144, 128), db = sdesc(smem_u32(W1), 128, 512);
                // issuer q takes tiles q, q + 4, ...; the tiles' accumulators are
                // independent, so consecutive MMAs go to different tiles and a
                // tile's accumulation chain does not stall the pipe
                for (int t = q; t < T1; t += 4) mma_bf16(tmem + 16 * t, da + (uint64_t)(t * 128), db, id, false);
                for (int t = q; t < T1; t += 4) mma_bf16(tmem + 16 * t, da + (uint64_t)(t * 128 + 18), db + 16, id, true);
            })) { failed = true; break; }
        CNN_PH(2);
        // epilogue: the 7 x 7 window -> conv2 input planes; a warp takes two
        // tiles (32 accumulator columns) of its lane quadrant per load
        for (int t0 = 2 * sub; t0 < T1; t0 += 8) {
            uint32_t v[32];
            tmem_ld32_nowait(tmem + lane_off + 16 * t0, v);
            tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int t = t0 + u;
                const int r = t * 128 + 32 * quad + lane;
                const int pp = r / 81, pos = r % 81, yy = pos / 9, xx = pos % 9;
                if (t < T1 && pp < FP && yy < 7 && xx < 7) {
                    uint4 lo, hi;
                    relu_bf16x16(v + 16 * u, SB + Q::b1, &lo, &hi);
                    const int o = pp * 49 + yy * 7 + xx;
                    reinterpret_cast<uint4 *>(X)[o] = lo;
                    reinterpret_cast<uint4 *>(X + (size_t)P1_ROWS * 16)[o] = hi;
                }
            }
        }
        CNN_PH(3);
        // ---- conv2: one MMA per tap (16 channels = the two planes) ----
        if (!run_layer([&](int q) {
                const uint32_t id = idesc_bf16(16);
                const uint64_t da = sdesc(xs, P1_ROWS * 16, 128), db = sdesc(smem_u32(W2), 128, 18 * 128);
#pragma unroll
                for (int k = 0; k < 9; ++k)
                    for (int t = q; t < T2; t += 4)
                        mma_bf16(tmem + 16 * t, da + (uint64_t)(t * 128 + (k / 3) * 7 + k % 3), db + 16 * k, id, k > 0);
            })) { failed = true; break; }
        CNN_PH(4);
        for (int t0 = 2 * sub; t0 < T2; t0 += 8) {
            uint32_t v[32];
            tmem_ld32_nowait(tmem + lane_off + 16 * t0, v);
            tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int t = t0 + u;
                const int r = t * 128 + 32 * quad + lane;
                const int pp = r / 49, pos = r % 49, yy = pos / 7, xx = pos % 7;
                if (t < T2 && pp < FP && yy < 5 && xx < 5) {
                    uint4 lo, hi;
                    relu_bf16x16(v + 16 * u, SB + Q::b2, &lo, &hi);
                    const int o = pp * 25 + yy * 5 + xx;
                    reinterpret_cast<uint4 *>(X)[o] = lo;
                    reinterpret_cast<uint4 *>(X + (size_t)P2_ROWS * 16)[o] = hi;
                }
            }
        }
        CNN_PH(5);
        // ---- conv3 ----
        if (!run_layer([&](int q) {
                const uint32_t id = idesc_bf16(32);
                const uint64_t da = sdesc(xs, P2_ROWS * 16, 128), db = sdesc(smem_u32(W3), 128, 18 * 128);
#pragma unroll
                for (int k = 0; k < 9; ++k)
                    for (int t = q; t < T3; t += 4)
                        mma_bf16(tmem + 32 * t, da + (uint64_t)(t * 128 + (k / 3) * 5 + k % 3), db + 16 * k, id, k > 0);
            })) { failed = true; break; }
        CNN_PH(6);
        // epilogue: the 3 x 3 window -> fc1 input, one row per patch, plane (pos * 4 + channel / 8)
        for (int t = sub; t < T3; t += 4) {
            uint32_t v[32];
            tmem_ld32_nowait(tmem + lane_off + 32 * t, v);
            tmem_wait_ld();
            const int r = t * 128 + 32 * quad + lane;
            const int pp = r / 25, pos = r % 25, yy = pos / 5, xx = pos % 5;
            if (pp < FP && yy < 3 && xx < 3) {
                uint4 a0, a1, a2, a3;
                relu_bf16x16(v, SB + Q::b3, &a0, &a1);
                relu_bf16x16(v + 16, SB + Q::b3 + 16, &a2, &a3);
                const int j = (yy * 3 + xx) * 4;
                *reinterpret_cast<uint4 *>(X + (size_t)(j + 0) * PLB + 16 * pp) = a0;
                *reinterpret_cast<uint4 *>(X + (size_t)(j + 1) * PLB + 16 * pp) = a1;
                *reinterpret_cast<uint4 *>(X + (size_t)(j + 2) * PLB + 16 * pp) = a2;
                *reinterpret_cast<uint4 *>(X + (size_t)(j + 3) * PLB + 16 * pp) = a3;
            }
        }
        CNN_PH(7);
        // ---- fc1: 18 MMAs over K = 288 (rows past the group's patches are dropped) ----
        if (!run_layer([&](int q) {
                const uint32_t id = idesc_bf16(144);
                const uint64_t da = sdesc(xs, PLB, 128), db = sdesc(smem_u32(W4), 128, 36 * 128);
                // three accumulators (columns 0, 160, 320) over interleaved k
                // steps, summed in the epilogue: three short chains, one per
                // issuer (the fourth issues nothing)
                if (q < 3)
#pragma unroll
                    for (int k = q; k < 18; k += 3)
                        mma_bf16(tmem + 160 * q, da + (uint64_t)(2 * k * (PLB / 16)), db + 16 * k, id, k >= 3);
            })) { failed = true; break; }
        CNN_PH(8);
        {
            const int pp = 32 * quad + lane;
#pragma unroll 1
            for (int c0 = 32 * sub; c0 < 144; c0 += 128) {   // 32 columns of each of the three accumulators per wait
                uint32_t v[32], u[32], w[32];
                tmem_ld32_nowait(tmem + lane_off + c0, v);
                tmem_ld32_nowait(tmem + lane_off + 160 + c0, u);
                tmem_ld32_nowait(tmem + lane_off + 320 + c0, w);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    v[j] = __float_as_uint(__uint_as_float(v[j]) + __uint_as_float(u[j]) + __uint_as_float(w[j]));
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = c0 + 16 * h;
                    if (c < 144 && pp < FP) {
                        uint4 lo, hi;
                        relu_bf16x16(v + 16 * h, SB + Q::b4 + c, &lo, &hi);
                        *reinterpret_cast<uint4 *>(X + (size_t)(c / 8) * PLB + 16 * pp) = lo;
                        *reinterpret_cast<uint4 *>(X + (size_t)(c / 8 + 1) * PLB + 16 * pp) = hi;
                    }
                }
            }
        }
        CNN_PH(9);
        // ---- fc2: 9 MMAs over K = 144, fp32 outputs ----
        if (!run_layer([&](int q) {
                const uint32_t id = idesc_bf16(16);
                const uint64_t da = sdesc(xs, PLB, 128), db = sdesc(smem_u32(W5), 128, 18 * 128);
                if (q < 3)
#pragma unroll
                    for (int k = q; k < 9; k += 3)
                        mma_bf16(tmem + 16 * q, da + (uint64_t)(2 * k * (PLB / 16)), db + 16 * k, id, k >= 3);
            })) { failed = true; break; }
        CNN_PH(10);
        if (sub == 0) {
            uint32_t v[32], u[16];
            tmem_ld32_nowait(tmem + lane_off, v);        // accumulators 0 and 1
            tmem_ld16(tmem + lane_off + 32, u);          // accumulator 2 (and the wait)
            const int pp = 32 * quad + lane;
            const long long row = g * FP + pp;
            if (pp < FP && row < n) {
#pragma unroll
                for (int j = 0; j < NOUT; ++j)
                    out[row * NOUT + j] = __uint_as_float(v[j]) + __uint_as_float(v[16 + j]) + __uint_as_float(u[j]) +
                                          SB[Q::b5 + j];
            }
        }
        CNN_PH(11);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    if (failed && tid == 0) atomicOr(status, tpxk::ST_DEVTIMEOUT);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

int launch_fused_cnn(tpx_ctx *c, const __nv_bfloat16 *x, long long n, const __nv_bfloat16 *wt, const float *bias,
                     float *out) {
    if (ck(cudaFuncSetAttribute(k_cnn_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FUSED_SMEM))) return TPX_ECUDA;
    const long long groups = (n + FP - 1) / FP;
    long long grid = c->num_sms;   // one CTA per SM: its shared memory and all of tensor memory
    if (grid > groups) grid = groups;
    k_cnn_fused<<<(unsigned)grid, CNN_THREADS, FUSED_SMEM, c->stream>>>(x, n, wt, bias, out, &c->ctl->status);
    return ck(cudaGetLastError()) ? TPX_ECUDA : TPX_OK;
}

}  // namespace tpxc

using namespace tpxc;

extern "C" {

int64_t tpx_cnn_params(void) { return NPARAM; }
int64_t tpx_cnn_work_floats(int64_t n) { return n > 0 ? n * kWork : 0; }

int tpx_cnn_forward(tpx_ctx *c, const float *d_params, const float *d_x, int64_t n, float *d_work, float *d_out) {
    if (!c || !d_params || n < 0 || (n > 0 && (!d_x || !d_work || !d_out)) || n > (1LL << 22)) return TPX_EINVAL;
    if (n == 0) return TPX_OK;
    Work w(d_work, n);
    int rc = forward32(c->stream, d_params, d_x, n, w);
    if (rc) return rc;
    return ck(cudaMemcpyAsync(d_out, w.out, sizeof(float) * NOUT * (size_t)n, cudaMemcpyDeviceToDevice, c->stream))
               ? TPX_ECUDA : TPX_OK;
}

int tpx_cnn_train_step(tpx_ctx *c, float *d_params, float *d_adam_m, float *d_adam_v, float *d_grad, int64_t step,
                       const float *d_x, const float *d_y, int64_t n, float lr, float offset_weight, float *d_work,
                       float *d_loss) {
    if (!c || !d_params || !d_adam_m || !d_adam_v || !d_grad || step < 1 || !d_x || !d_y || n < 1 || !d_work ||
        !d_loss || n > (1LL << 20))
        return TPX_EINVAL;
    cudaStream_t s = c->stream;
    Work w(d_work, n);
    int rc = forward32(s, d_params, d_x, n, w);
    if (rc) return rc;
    if (ck(cudaMemsetAsync(d_loss, 0, 4, s)) || ck(cudaMemsetAsync(d_grad, 0, sizeof(float) * NPARAM, s))) return TPX_ECUDA;
    rc = tpxr_loss(s, w.out, d_y, (int)n, offset_weight, w.dout, d_loss);
    if (rc) return rc;
    // fc2, fc1
    layer_back(s, d_params, d_grad, layer_of(4), w.a4, w.dout, n, w.d4);
    k_relu_back<<<grid_for(n * 144), 256, 0, s>>>(w.d4, w.a4, n * 144);
    layer_back(s, d_params, d_grad, layer_of(3), w.x4, w.d4, n, w.dx4);
    k_col2im<<<grid_for(n * 9 * 32), 256, 0, s>>>(w.dx4, n, 32, 3, 1, 3, w.d3);
    // conv3, conv2, conv1
    k_relu_back<<<grid_for(n * 9 * 32), 256, 0, s>>>(w.d3, w.a3, n * 9 * 32);
    layer_back(s, d_params, d_grad, layer_of(2), w.x3, w.d3, n * 9, w.dx3);
    k_col2im<<<grid_for(n * 25 * 16), 256, 0, s>>>(w.dx3, n, 16, 5, 3, 3, w.d2);
    k_relu_back<<<grid_for(n * 25 * 16), 256, 0, s>>>(w.d2, w.a2, n * 25 * 16);
    layer_back(s, d_params, d_grad, layer_of(1), w.x2, w.d2, n * 25, w.dx2);
    k_col2im<<<grid_for(n * 49 * 16), 256, 0, s>>>(w.dx2, n, 16, 7, 5, 3, w.d1);
    k_relu_back<<<grid_for(n * 49 * 16), 256, 0, s>>>(w.d1, w.a1, n * 49 * 16);
    layer_back(s, d_params, d_grad, layer_of(0), w.x1, w.d1, n * 49, nullptr);
    if (ck(cudaGetLastError())) return TPX_ECUDA;
    return tpxr_adam(s, d_params, d_grad, d_adam_m, d_adam_v, NPARAM, lr, step);
}

int64_t tpx_cnn_packed_bytes(void) { return (int64_t)Packed::bytes; }

int tpx_cnn_pack(tpx_ctx *c, const float *d_params, void *d_packed) {
    if (!c || !d_params || !d_packed || (reinterpret_cast<uintptr_t>(d_packed) & 255)) return TPX_EINVAL;
    __nv_bfloat16 *wt = static_cast<__nv_bfloat16 *>(d_packed);
    float *bias = reinterpret_cast<float *>(static_cast<char *>(d_packed) + Packed::boff);
    k_cnn_pack<<<grid_for((long long)Packed::wend + (long long)Packed::bend), 256, 0, c->stream>>>(d_params, wt, bias);
    return ck(cudaGetLastError()) ? TPX_ECUDA : TPX_OK;
}

int64_t tpx_cnn_infer_work_bytes(int64_t n) { return n > 0 ? 256 : 0; }

int tpx_debug_cnn_phase_times(uint64_t *h_cycles, int clear) {
    if (!h_cycles) return TPX_EINVAL;
#ifdef TPX_PHASE_TIMING
    if (cudaDeviceSynchronize() != cudaSuccess) return TPX_ECUDA;
    cudaError_t e = cudaMemcpyFromSymbol(h_cycles, g_cnn_phase, 16 * 8);
    if (e == cudaSuccess && clear) {
        static const unsigned long long zero[16] = {0};
        e = cudaMemcpyToSymbol(g_cnn_phase, zero, 16 * 8);
    }
    return e == cudaSuccess ? TPX_OK : TPX_ECUDA;
#else
    (void)clear;
    for (int i = 0; i < 16; ++i) h_cycles[i] = 0;
    return TPX_EUNSUPPORTED;
#endif
}

int tpx_cnn_infer(tpx_ctx *c, const void *d_packed, const uint16_t *d_x, int64_t n, void *d_work, float *d_out) {
    if (!c || n < 0 || (n > 0 && (!d_packed || !d_x || !d_out)) || n > (1LL << 30)) return TPX_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_packed) & 255) || (reinterpret_cast<uintptr_t>(d_x) & 15)) return TPX_EINVAL;
    (void)d_work;
    if (n == 0) return TPX_OK;
    const __nv_bfloat16 *wt = static_cast<const __nv_bfloat16 *>(d_packed);
    const float *bias = reinterpret_cast<const float *>(static_cast<const char *>(d_packed) + Packed::boff);
    return launch_fused_cnn(c, reinterpret_cast<const __nv_bfloat16 *>(d_x), n, wt, bias, d_out);
}

}  // extern "C"
