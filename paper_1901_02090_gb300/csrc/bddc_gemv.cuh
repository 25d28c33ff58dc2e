// Warp GEMV y = M x for one subdomain operator (S, F), n x n, input-major
// (entry (o, j) at M[j*n + o]), with every output written by exactly one
// lane through a callback.
//
// Outputs come in passes of 32, lane l taking output o0 + l over all n inputs
// (the loads of a pass are consecutive across lanes: coalesced).  The last
// r = n mod 32 outputs would leave 32 - r lanes idle in a plain pass; they
// are split instead: with R the power of two >= r and G = 32 / R groups, lane
// l takes output (l mod R) over the G-th part l / R of the inputs, and the G
// partial sums are added by xor shuffles.  For the n = 40 of a 10 x 10-cell
// subdomain a lane then does 40 + 10 accumulation steps instead of 80.
// Loads are issued 8 at a time ahead of their products.
//
// Included by bddc_kernels.cu inside namespace bddc (after WarpSm and the
// double-float arithmetic).
#pragma once

// accumulators: FP64 on x, FP32 on xh, FP32 pair on (xh, xl)
template <class T>
struct GAcc;
template <>
struct GAcc<double> {
    using value_type = double;
    double s = 0.0;
    __device__ __forceinline__ void add(double m, const WarpSm& w, int j) { s = fma(m, w.x[j], s); }
    __device__ __forceinline__ void shfl_add(int off) { s += __shfl_xor_sync(0xffffffffu, s, off); }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct GAcc<float> {
    using value_type = double;
    float s = 0.0f;
    __device__ __forceinline__ void add(float m, const WarpSm& w, int j) { s = fmaf(m, w.xh[j], s); }
    __device__ __forceinline__ void shfl_add(int off) { s += __shfl_xor_sync(0xffffffffu, s, off); }
    __device__ __forceinline__ double value() const { return (double)s; }
};
template <>
struct GAcc<float2> {
    using value_type = float2;
    float h = 0.0f, l = 0.0f;
    __device__ __forceinline__ void add(float2 m, const WarpSm& w, int j) { dd_acc(h, l, m, w.xh[j], w.xl[j]); }
    __device__ __forceinline__ void shfl_add(int off) {
        const float2 o = make_float2(__shfl_xor_sync(0xffffffffu, h, off), __shfl_xor_sync(0xffffffffu, l, off));
        const float2 v = dd_add(dd_quick(h, l), o);
        h = v.x;
        l = v.y;
    }
    __device__ __forceinline__ float2 value() const { return dd_quick(h, l); }
};

// a += sum_{j0 <= j < j1} M[j*n + o] x_j
template <class T>
__device__ __forceinline__ void gemv_column(const T* __restrict__ M, int n, const WarpSm& w, int o, int j0, int j1,
                                            GAcc<T>& a) {
    int j = j0;
    for (; j + 8 <= j1; j += 8) {
        T A[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) A[t] = __ldg(M + (int64_t)(j + t) * n + o);
#pragma unroll
        for (int t = 0; t < 8; ++t) a.add(A[t], w, j + t);
    }
    for (; j < j1; ++j) a.add(__ldg(M + (int64_t)j * n + o), w, j);
}

// out(o, y_o) for the outputs o = ob..oe-1 of the n x n operator, each o on
// one lane; called by the whole warp
template <class T, class Out>
__device__ __forceinline__ void gemv_warp_range(const T* __restrict__ M, int n, int ob, int oe, const WarpSm& w,
                                                Out&& out) {
    const int l = threadIdx.x & 31;
    const int full = ob + ((oe - ob) & ~31);
    for (int o0 = ob; o0 < full; o0 += 32) {
        GAcc<T> a;
        gemv_column(M, n, w, o0 + l, 0, n, a);
        out(o0 + l, a.value());
    }
    const int r = oe - full;
    if (r == 0) return;
    int R = 1;
    while (R < r) R <<= 1;
    const int G = 32 / R;
    const int e = l & (R - 1), g = l / R;
    const int o = full + (e < r ? e : r - 1);  // lanes past r repeat a valid column; their sums are dropped
    GAcc<T> a;
    gemv_column(M, n, w, o, (n * g) / G, (n * (g + 1)) / G, a);
    for (int off = R; off < 32; off <<= 1) a.shfl_add(off);
    if (g == 0 && e < r) out(o, a.value());
}

// out(o, y_o) for o = 0..n-1
template <class T, class Out>
__device__ __forceinline__ void gemv_warp(const T* __restrict__ M, int n, const WarpSm& w, Out&& out) {
    gemv_warp_range(M, n, 0, n, w, static_cast<Out&&>(out));
}
