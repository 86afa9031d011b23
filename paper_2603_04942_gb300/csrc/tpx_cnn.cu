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
// back from the column gradients). Inference: each layer is an implicit GEMM
// on the fifth-generation tensor cores -- the im2col tile of 128 output
// positions is gathered straight into shared memory, one thread issues
// tcgen05.mma (bf16 operands, fp32 accumulator in tensor memory), the
// epilogue reads the accumulator with tcgen05.ld, adds the bias, applies the
// ReLU and rounds the activation to bf16 for the next layer.
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

template <int CIN, int HIN, int N, int HO, int KK, int KP, bool IN_CHW, bool OUT_F32, int COUT>
struct TcLayer {
    static constexpr int K = CIN * KK * KK;   // real reduction length
    static constexpr int ROWS = HO * HO;      // output positions per patch
    static constexpr int TCOLS = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));   // TMEM columns
    // layers with several output positions per patch stage the inputs of the
    // tile's patches in shared memory first (coalesced), then gather from there
    static constexpr bool STAGE = HO > 1;
    static constexpr int PIN = CIN * HIN * HIN;                      // input elements per patch
    static constexpr int PPT = STAGE ? (127 + ROWS - 1) / ROWS + 1 : 0;   // patches a tile can span
    static constexpr size_t A_BYTES = (size_t)128 * KP * 2, B_BYTES = (size_t)N * KP * 2;
    static constexpr size_t IN_BYTES = (((size_t)PPT * PIN * 2 + 15) / 16) * 16;
    static constexpr size_t SMEM = A_BYTES + B_BYTES + IN_BYTES + 64 + 1024;   // + barrier, TMEM address, alignment
    static_assert(KP % 16 == 0 && KP >= K && N % 16 == 0 && N >= 16 && N <= 256 && COUT <= N, "tcgen05 shape");
};

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

template <int CIN, int HIN, int N, int HO, int KK, int KP, bool IN_CHW, bool OUT_F32, int COUT>
__global__ void __launch_bounds__(128) k_conv_tc(const __nv_bfloat16 *__restrict__ in, long long n_rows,
                                                 const __nv_bfloat16 *__restrict__ w, const float *__restrict__ bias,
                                                 void *__restrict__ out, unsigned *status) {
    using G = TcLayer<CIN, HIN, N, HO, KK, KP, IN_CHW, OUT_F32, COUT>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *As = base;
    unsigned char *Bs = base + G::A_BYTES;
    __nv_bfloat16 *Sin = reinterpret_cast<__nv_bfloat16 *>(Bs + G::B_BYTES);
    uint64_t *bar = reinterpret_cast<uint64_t *>(Bs + G::B_BYTES + G::IN_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // the weights, once: [N][KP] bf16 rows into the core-matrix layout
    for (int i = tid; i < N * (KP / 8); i += 128) {
        const int r = i / (KP / 8), c = i % (KP / 8);
        *reinterpret_cast<uint4 *>(Bs + core_off(r, c * 8, KP)) = *reinterpret_cast<const uint4 *>(w + (size_t)r * KP + c * 8);
    }
    if (tid == 0) mbar_init(smem_u32(bar), 1);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)G::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t a_base = smem_u32(As), b_base = smem_u32(Bs);
    constexpr uint32_t SBO = (KP / 8) * 128;
    uint32_t phase = 0;

    const long long tiles = (n_rows + 127) / 128;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        bool failed = false;
        // ---- the im2col tile: 128 output positions x KP reduction columns ----
        const long long r0 = tile * 128;
        const long long n_pat = (n_rows + G::ROWS - 1) / G::ROWS;
        const long long pf = r0 / G::ROWS;   // the tile's first patch
        if (G::STAGE) {   // the inputs of the tile's patches, coalesced, into shared memory
            const long long pl = min(n_pat, (r0 + 127) / G::ROWS + 1);
            const int elems = (int)((pl - pf) * G::PIN);
            const __nv_bfloat16 *src = in + pf * G::PIN;
            if (G::PIN % 8 == 0) {
                for (int i = tid; i < elems / 8; i += 128) cp16(Sin + 8 * i, src + 8 * i, true);
            } else {      // PIN is even: 4-byte words
                for (int i = tid; i < elems / 2; i += 128) cp4(Sin + 2 * i, src + 2 * i);
            }
            cp_wait_all();
            __syncthreads();
        }
        if (G::STAGE) {   // one thread per row: the taps' offsets are compile-time constants
            const int r = tid;
            const long long row = r0 + r;
            const bool valid = row < n_rows;
            const int p = valid ? (int)(row / G::ROWS - pf) : 0;
            const int pos = valid ? (int)(row % G::ROWS) : 0, oy = pos / HO, ox = pos % HO;
            unsigned char *arow = As + core_off(r, 0, KP);
            if (IN_CHW) {   // conv1: channel-major patch rows of 162, two k at a time
                const __nv_bfloat16 *src = Sin + p * G::PIN + oy * HIN + ox;
#pragma unroll
                for (int k = 0; k < KP; k += 2) {
                    __nv_bfloat16 v[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int kk = k + u, ci = kk / (KK * KK), t = kk % (KK * KK);
                        v[u] = (valid && kk < G::K) ? src[ci * HIN * HIN + (t / KK) * HIN + (t % KK)] : __float2bfloat16_rn(0.f);
                    }
                    *reinterpret_cast<__nv_bfloat162 *>(arow + (((k >> 3) << 7) + ((k & 7) << 1))) = __halves2bfloat162(v[0], v[1]);
                }
            } else {        // channel-minor activations: 8 channels of a tap per 16-byte chunk
                static_assert(IN_CHW || CIN % 8 == 0, "16-byte gathers");
                const __nv_bfloat16 *src = Sin + p * G::PIN + (oy * HIN + ox) * CIN;
#pragma unroll
                for (int c8 = 0; c8 < KP; c8 += 8) {
                    const int t = c8 / CIN, ci = c8 % CIN;
                    uint4 v = make_uint4(0, 0, 0, 0);
                    if (valid && c8 < G::K) v = *reinterpret_cast<const uint4 *>(src + ((t / KK) * HIN + (t % KK)) * CIN + ci);
                    *reinterpret_cast<uint4 *>(arow + ((c8 >> 3) << 7)) = v;
                }
            }
        } else {        // one output position per patch: the row is the patch's activations, copied
            for (int i = tid; i < 128 * (KP / 8); i += 128) {
                const int r = i / (KP / 8), c8 = (i % (KP / 8)) * 8;
                const long long row = r0 + r;
                const bool ok = row < n_rows && c8 < G::K;
                cp16(As + core_off(r, c8, KP), ok ? in + row * G::K + c8 : in, ok);
            }
            cp_wait_all();
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        // ---- one thread issues the MMAs over the reduction, then commits ----
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int s = 0; s < KP / 16; ++s) {
                const uint64_t ad = sdesc(a_base + 256 * s, 128, SBO);
                const uint64_t bd = sdesc(b_base + 256 * s, 128, SBO);
                const uint32_t acc = s > 0 ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc_bf16(N)), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                         : "memory");
        }
        // ---- wait for the accumulator (bounded; a wait that runs out sets the
        // status and every thread leaves the loop, then frees the TMEM) ----
        long long spins = 0;
        while (!mbar_try_wait(smem_u32(bar), phase)) {
            if (++spins > kSpin) { failed = true; break; }
        }
        if (__syncthreads_or(failed ? 1 : 0)) {
            if (tid == 0) atomicOr(status, tpxk::ST_DEVTIMEOUT);
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // ---- epilogue: warp w reads accumulator lanes 32w..32w+31 (its rows) ----
        const long long row = r0 + 32 * warp + lane;
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t v[16];
            const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < n_rows) {
                if (OUT_F32) {
                    float *o = reinterpret_cast<float *>(out) + row * COUT;
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (c0 + j < COUT) o[c0 + j] = __uint_as_float(v[j]) + bias[c0 + j];
                } else {
                    __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(out) + row * COUT + c0;
                    uint32_t pk[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float lo = fmaxf(__uint_as_float(v[2 * j]) + bias[c0 + 2 * j], 0.f);
                        const float hi = fmaxf(__uint_as_float(v[2 * j + 1]) + bias[c0 + 2 * j + 1], 0.f);
                        __nv_bfloat162 b2 = __floats2bfloat162_rn(lo, hi);
                        pk[j] = *reinterpret_cast<uint32_t *>(&b2);
                    }
                    reinterpret_cast<uint4 *>(o)[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    reinterpret_cast<uint4 *>(o)[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();   // the accumulator and the A tile are free again
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)G::TCOLS)
                     : "memory");
}

// packed inference weights: per layer [N][KP] bf16 with column k = tap * cin +
// ci (8 channels of a tap per 16-byte chunk; conv1: ci * 9 + tap), zero
// padded; then the biases (fp32, padded to N)
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
        if (r < C.cout && k < K) {
            int ci, t;
            if (L == 0) { ci = k / kk2; t = k % kk2; }   // conv1 gathers channel-major
            else { t = k / C.cin; ci = k % C.cin; }
            v = P[C.ow + (long long)r * K + ci * kk2 + t];   // [cout][cin][tap]
        }
        wt[i] = __float2bfloat16_rn(v);
    }
}

template <int CIN, int HIN, int N, int HO, int KK, int KP, bool IN_CHW, bool OUT_F32, int COUT>
int launch_tc(tpx_ctx *c, const __nv_bfloat16 *in, long long n_rows, const __nv_bfloat16 *w, const float *bias, void *out) {
    using G = TcLayer<CIN, HIN, N, HO, KK, KP, IN_CHW, OUT_F32, COUT>;
    auto kern = k_conv_tc<CIN, HIN, N, HO, KK, KP, IN_CHW, OUT_F32, COUT>;
    if (ck(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM))) return TPX_ECUDA;
    // CTAs per SM: by shared memory (227 KB, 1 KB reserved per CTA), by
    // threads (16 of 128), and by tensor memory (each holds TCOLS of 512 columns)
    int per_sm = (int)((227 * 1024) / (G::SMEM + 1024));
    if (per_sm > 16) per_sm = 16;
    if (per_sm > 512 / G::TCOLS) per_sm = 512 / G::TCOLS;
    if (per_sm < 1) per_sm = 1;
    const long long tiles = (n_rows + 127) / 128;
    long long grid = (long long)c->num_sms * per_sm;
    if (grid > tiles) grid = tiles;
    if (grid < 1) return TPX_OK;
    kern<<<(unsigned)grid, 128, G::SMEM, c->stream>>>(in, n_rows, w, bias, out, &c->ctl->status);
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

int64_t tpx_cnn_infer_work_bytes(int64_t n) {
    if (n <= 0) return 0;
    return n * (int64_t)(49 * 16 + 25 * 16 + 9 * 32 + 144) * 2 + 1024;
}

int tpx_cnn_infer(tpx_ctx *c, const void *d_packed, const uint16_t *d_x, int64_t n, void *d_work, float *d_out) {
    if (!c || n < 0 || (n > 0 && (!d_packed || !d_x || !d_work || !d_out)) || n > (1LL << 30)) return TPX_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_packed) & 255) || (reinterpret_cast<uintptr_t>(d_x) & 15) ||
        (reinterpret_cast<uintptr_t>(d_work) & 15))
        return TPX_EINVAL;
    if (n == 0) return TPX_OK;
    using Q = Packed;
    const __nv_bfloat16 *wt = static_cast<const __nv_bfloat16 *>(d_packed);
    const float *bias = reinterpret_cast<const float *>(static_cast<const char *>(d_packed) + Q::boff);
    __nv_bfloat16 *a1 = static_cast<__nv_bfloat16 *>(d_work);
    __nv_bfloat16 *a2 = a1 + n * 49 * 16, *a3 = a2 + n * 25 * 16, *a4 = a3 + n * 9 * 32;
    const __nv_bfloat16 *x = reinterpret_cast<const __nv_bfloat16 *>(d_x);
    int rc;
    if ((rc = launch_tc<2, 9, 16, 7, 3, 32, true, false, 16>(c, x, n * 49, wt + Q::w1, bias + Q::b1, a1))) return rc;
    if ((rc = launch_tc<16, 7, 16, 5, 3, 144, false, false, 16>(c, a1, n * 25, wt + Q::w2, bias + Q::b2, a2))) return rc;
    if ((rc = launch_tc<16, 5, 32, 3, 3, 144, false, false, 32>(c, a2, n * 9, wt + Q::w3, bias + Q::b3, a3))) return rc;
    if ((rc = launch_tc<32, 3, 144, 1, 3, 288, false, false, 144>(c, a3, n, wt + Q::w4, bias + Q::b4, a4))) return rc;
    return launch_tc<144, 1, 16, 1, 1, 144, false, true, NOUT>(c, a4, n, wt + Q::w5, bias + Q::b5, d_out);
}

}  // extern "C"
