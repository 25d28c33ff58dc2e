// L2 residency hints for the loads of the solve kernel.
//
// Per iteration the coarse phase streams the flux columns of every
// instance's dense coarse inverse once -- the largest read of an iteration,
// larger than L2 for a batch of tens of instances.  Those loads carry an
// evict_first policy so that the streamed rows do not displace the
// per-subdomain vectors and index arrays that the following phases re-read.
// Included by bddc_kernels.cu inside namespace bddc.
#pragma once

__device__ __forceinline__ uint64_t l2_stream_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// read-only loads with an L2 cache policy
__device__ __forceinline__ double ld_hint(const double* ptr, uint64_t pol) {
    double v;
    asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_hint(const float* ptr, uint64_t pol) {
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ float2 ld_hint(const float2* ptr, uint64_t pol) {
    float2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(ptr), "l"(pol));
    return v;
}

// L2 prefetch of the 128-byte line holding ptr.  A prefetch only warms L2:
// the data still arrives through the normal loads, which then hit L2
// instead of waiting for DRAM.  The sparse coarse sweeps use it for a
// unit's matrix rows, whose loads it issues in batches of 8 (the kernel's
// register cap).  (A bulk prefetch of the subdomain operator blocks at the
// start of a unit was measured slower: their loads follow at once.)
__device__ __forceinline__ void prefetch_l2_line(const void* ptr) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}
// the lines of n consecutive doubles from ptr (n <= 32): elements 0, 16 and
// n - 1 lie on every line the range touches
__device__ __forceinline__ void prefetch_l2_row32(const double* ptr, int n) {
    if (n <= 0) return;
    prefetch_l2_line(ptr);
    if (n > 16) prefetch_l2_line(ptr + 16);
    prefetch_l2_line(ptr + n - 1);
}
