// tpx_common.cuh -- device helpers shared by the fused kernel and the
// general (global-memory) path: packet decoding and the associative ToA
// unwrap chains.
//
// Unwrap (Sec. IV.A): per stream (pixels, TDCs) in stream order, a step from
// the previous raw value down by more than the threshold adds one wrap period
// to everything after it and a step up by more than it removes one. A
// stretch of the stream is summarised by (count, first raw, last raw, sum of
// the steps inside it); two consecutive stretches combine by adding their sums
// plus the step between the first's last and the second's first value, which
// is associative, so the chain state at any position follows from a scan.
#pragma once

#include <cstdint>

#include "tpx_fused.cuh"

namespace tpxk {

__device__ __forceinline__ long long pix_raw(uint64_t w) {
    long long coarse = (long long)(((w & 0xFFFFull) << 14) | ((w >> 30) & 0x3FFFull));
    long long ftoa = (long long)((w >> 16) & 0xFull);
    return (coarse * 16 - ftoa) & (kPixPeriod - 1);
}
__device__ __forceinline__ long long tdc_raw(uint64_t w) {
    return (long long)(((w >> 9) & ((1ull << 35) - 1)) << 1);
}
__device__ __forceinline__ int pix_x(uint64_t w) { return (int)(2 * ((w >> 53) & 0x7F) + (((w >> 44) & 7) >> 2)); }
__device__ __forceinline__ int pix_y(uint64_t w) { return (int)(4 * ((w >> 47) & 0x3F) + ((w >> 44) & 3)); }
__device__ __forceinline__ int pix_tot(uint64_t w) { return (int)((w >> 20) & 0x3FF); }

__device__ __forceinline__ long long jump(long long d, long long thr) { return d < -thr ? 1 : (d > thr ? -1 : 0); }

__device__ __forceinline__ GChain chain_id() { GChain c; c.n = 0; c.first = 0; c.last = 0; c.sum = 0; return c; }
__device__ __forceinline__ GAgg agg_id() { GAgg a; a.pix = chain_id(); a.tdc = chain_id(); return a; }

// associative combine of two consecutive stretches of one unwrap chain
__device__ __forceinline__ GChain ccomb(const GChain &a, const GChain &b, long long thr) {
    GChain c;
    c.n = a.n + b.n;
    c.first = a.n ? a.first : b.first;
    c.last = b.n ? b.last : a.last;
    c.sum = a.sum + b.sum + ((a.n && b.n) ? jump(b.first - a.last, thr) : 0);
    return c;
}
__device__ __forceinline__ GAgg acomb(const GAgg &a, const GAgg &b, long long tp, long long tt) {
    GAgg c;
    c.pix = ccomb(a.pix, b.pix, tp);
    c.tdc = ccomb(a.tdc, b.tdc, tt);
    return c;
}
__device__ __forceinline__ void chain_push(GChain &c, long long raw, long long thr) {
    if (c.n) c.sum += jump(raw - c.last, thr); else c.first = raw;
    c.last = raw;
    c.n += 1;
}

__device__ __forceinline__ GChain shfl_up_chain(const GChain &v, int o) {
    GChain u;
    u.n = __shfl_up_sync(0xffffffffu, v.n, o);
    u.first = __shfl_up_sync(0xffffffffu, v.first, o);
    u.last = __shfl_up_sync(0xffffffffu, v.last, o);
    u.sum = __shfl_up_sync(0xffffffffu, v.sum, o);
    return u;
}
__device__ __forceinline__ GAgg shfl_up_agg(const GAgg &v, int o) {
    GAgg u;
    u.pix = shfl_up_chain(v.pix, o);
    u.tdc = shfl_up_chain(v.tdc, o);
    return u;
}
__device__ __forceinline__ GAgg warp_incl_scan(GAgg v, int lane, long long tp, long long tt) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        GAgg u = shfl_up_agg(v, o);
        if (lane >= o) v = acomb(u, v, tp, tt);
    }
    return v;
}

// Sec. V.C centre of mass and ToT-weighted ToF from the exact integer
// moments: one reciprocal of S_tot, then products (each within a few ulp of
// the quotient; S_tot = 0 gives NaN, as 0/0 does)
__device__ __forceinline__ void com_from_moments(long long s_x, long long s_y, long long s_t, long long s_tot,
                                                 long long tof0, double *x, double *y, double *tof) {
    const double r = 1.0 / (double)s_tot;
    *x = (double)s_x * r;
    *y = (double)s_y * r;
    *tof = (double)tof0 + (double)s_t * r;
}

}  // namespace tpxk
