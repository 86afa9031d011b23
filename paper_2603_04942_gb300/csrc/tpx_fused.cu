// tpx_fused.cu -- fused single-pass TPX3 decode / unwrap / bin / cluster /
// centroid kernel for sm_103a.  See tpx_fused.cuh for the structure.
#include <cuda_runtime.h>

#include <atomic>
#include <climits>
#include <cstddef>
#include <cstdint>

#include "tpx_common.cuh"
#include "tpx_fused.cuh"

namespace tpxk {

constexpr int kAttrDevices = 64;   // devices whose kernel attributes are remembered

// 1024-thread CTAs, one per SM, 4096-packet tiles, 8192-position ranges
namespace geo_t4096 {
constexpr int NT = 1024, T = 4096, C = 8192, HB = 16384, MS = T + 16, MINB = 1;
#include "tpx_fused_body.cuh"
}  // namespace geo_t4096

// 512-thread CTAs, two per SM, 2048-packet tiles, 5120-position ranges (any
// shot of up to 3072 packets fits, wherever its trigger falls in the tile)
namespace geo_t2048 {
constexpr int NT = 512, T = 2048, C = 5120, HB = 8192, MS = T / 4 + 16, MINB = 2;
#include "tpx_fused_body.cuh"
}  // namespace geo_t2048

int fused_tile_packets(int geo) { return geo == GEO_T2048 ? geo_t2048::T : geo_t4096::T; }
int fused_threads(int geo) { return geo == GEO_T2048 ? geo_t2048::NT : geo_t4096::NT; }
int fused_range_capacity(int geo) { return geo == GEO_T2048 ? geo_t2048::C : geo_t4096::C; }
int fused_ctas_per_sm(int geo) { return geo == GEO_T2048 ? geo_t2048::MINB : geo_t4096::MINB; }
int fused_smem_bytes(int geo) { return geo == GEO_T2048 ? geo_t2048::smem_bytes() : geo_t4096::smem_bytes(); }
size_t fused_big_scratch_bytes(int geo) { return geo == GEO_T2048 ? geo_t2048::BR_STRIDE : geo_t4096::BR_STRIDE; }

cudaError_t launch_fused(const Params &p, int mode, int geo, int grid, cudaStream_t s, cudaEvent_t mid) {
    cudaError_t e = launch_unwrap_prepass(p, fused_tile_packets(geo), grid, s);
    if (e == cudaSuccess && mid) e = cudaEventRecord(mid, s);
    if (e != cudaSuccess) return e;
    return geo == GEO_T2048 ? geo_t2048::launch(p, mode, grid, s) : geo_t4096::launch(p, mode, grid, s);
}

}  // namespace tpxk

// Per-phase cycle counters of the instrumented build (-DTPX_PHASE_TIMING).
extern "C" int tpx_debug_phase_times(int tile_geometry, uint64_t *h_cycles, int clear) {
    if (!h_cycles || (tile_geometry != TPX_TILE_4096 && tile_geometry != TPX_TILE_2048)) return TPX_EINVAL;
#ifdef TPX_PHASE_TIMING
    const bool g2 = tile_geometry == TPX_TILE_2048;
    if (cudaDeviceSynchronize() != cudaSuccess) return TPX_ECUDA;
    cudaError_t e = g2 ? cudaMemcpyFromSymbol(h_cycles, tpxk::geo_t2048::g_phase, 32 * 8)
                       : cudaMemcpyFromSymbol(h_cycles, tpxk::geo_t4096::g_phase, 32 * 8);
    if (e == cudaSuccess && clear) {
        static const unsigned long long zero[32] = {0};
        e = g2 ? cudaMemcpyToSymbol(tpxk::geo_t2048::g_phase, zero, 32 * 8)
               : cudaMemcpyToSymbol(tpxk::geo_t4096::g_phase, zero, 32 * 8);
    }
    return e == cudaSuccess ? TPX_OK : TPX_ECUDA;
#else
    (void)clear;
    for (int i = 0; i < 32; ++i) h_cycles[i] = 0;
    return TPX_EUNSUPPORTED;
#endif
}
