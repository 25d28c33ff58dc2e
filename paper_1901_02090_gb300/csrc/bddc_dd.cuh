// Double-float ("FP32 pair") arithmetic: a value is hi + lo with two FP32,
// 48 significant bits, operated on with error-free FP32 transformations
// (Knuth's two-sum, Dekker's product via FMA).  Included by bddc_kernels.cu
// inside namespace bddc.
#pragma once

// All operations use explicitly rounded intrinsics so that no FMA contraction
// changes the error-free transformations.
__device__ __forceinline__ float2 dd_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 dd_quick(float a, float b) {
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 dd_add(float2 a, float2 b) {
    const float2 s = dd_two_sum(a.x, b.x);
    return dd_quick(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 dd_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 dd_sub(float2 a, float2 b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ float2 dd_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return dd_quick(p, e);
}
// a * sign, sign = +1 or -1 (exact)
__device__ __forceinline__ float2 dd_sign(float2 a, float sgn) { return sgn > 0.0f ? a : dd_neg(a); }
__device__ __forceinline__ float2 dd_of(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double dd_dbl(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ float2 dd_zero() { return make_float2(0.0f, 0.0f); }
// xor-butterfly sum: dd_add is commutative, so every lane gets the same bits
__device__ __forceinline__ float2 dd_warp_sum(float2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float2 t = make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
        v = dd_add(v, t);
    }
    return v;
}

// views of the work buffers as FP32 pairs (same 8-byte slots)
__device__ __forceinline__ float2* V2(double* p) { return reinterpret_cast<float2*>(p); }

// one compensated step of the FP32-pair dot product: (sh, sl) += a * (xh + xl)
__device__ __forceinline__ void dd_acc(float& sh, float& sl, float2 a, float xh, float xl) {
    const float pr = __fmul_rn(a.x, xh);
    float e = __fmaf_rn(a.x, xh, -pr);
    e = __fmaf_rn(a.x, xl, e);
    e = __fmaf_rn(a.y, xh, e);
    const float t = __fadd_rn(sh, pr);
    const float bp = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(pr, bp));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
}

