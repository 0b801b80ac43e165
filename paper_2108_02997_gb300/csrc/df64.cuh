// df64.cuh — the three value types the iteration kernels are written over.
//
//   double : native IEEE FP64 (runs on GB300's FP64 pipe, ~1/69 of FP32 rate)
//   float  : native FP32
//   df64   : an unevaluated sum hi + lo of two floats ("double-float"), about
//            48 significant bits, built only from FP32 operations.
//
// df64 uses the error-free transformations TwoSum (Knuth, TAOCP vol. 2,
// 4.2.2), Fast-TwoSum (Dekker 1971) and the FMA-based TwoProduct, as in the
// double-word arithmetic of Joldes, Muller and Popescu (ACM TOMS 2017). The
// explicit __fadd_rn/__fmul_rn/__fmaf_rn intrinsics keep the compiler from
// contracting or reassociating the steps that recover rounding errors.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct __align__(8) df64 {
    float hi, lo;
};

// ---------------------------------------------------------------- error-free transforms
__device__ __forceinline__ df64 ef_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df64 ef_fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

// ---------------------------------------------------------------- df64 arithmetic
__device__ __forceinline__ df64 df_make(float hi) { return {hi, 0.0f}; }

// Accurate sum of two double-floats (cancellation-safe).
__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
    df64 s = ef_two_sum(a.hi, b.hi);
    df64 t = ef_two_sum(a.lo, b.lo);
    float c = __fadd_rn(s.lo, t.hi);
    df64 v = ef_fast_two_sum(s.hi, c);
    float w = __fadd_rn(t.lo, v.lo);
    return ef_fast_two_sum(v.hi, w);
}
__device__ __forceinline__ df64 df_neg(df64 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df64 df_sub(df64 a, df64 b) { return df_add(a, df_neg(b)); }

// Sum of two non-negative double-floats (no cancellation possible).
__device__ __forceinline__ df64 df_add_pos(df64 a, df64 b) {
    df64 s = ef_two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return ef_fast_two_sum(s.hi, e);
}

// Product of two double-floats (FMA-based TwoProduct for the leading term).
__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ef_fast_two_sum(p, e);
}

// Division of a double-float by a positive integer d (d < 2^31).
__device__ __forceinline__ df64 df_div_int(df64 x, int32_t d) {
    float dh = __int2float_rn(d);
    float dl = __int2float_rn(d - __float2int_rn(dh));       // exact: |d - dh| <= 64
    float q1 = __fdiv_rn(x.hi, dh);
    // remainder x - q1 * (dh + dl), carried in double-float
    float p = __fmul_rn(q1, dh);
    float pe = __fmaf_rn(q1, dh, -p);
    df64 r = ef_two_sum(x.hi, -p);
    float rl = __fadd_rn(__fsub_rn(__fadd_rn(r.lo, x.lo), pe), -__fmul_rn(q1, dl));
    float rr = __fadd_rn(r.hi, rl);
    float q2 = __fdiv_rn(rr, dh);
    return ef_fast_two_sum(q1, q2);
}

__device__ __forceinline__ df64 df_abs(df64 a) { return a.hi < 0.0f ? df_neg(a) : a; }
__device__ __forceinline__ bool df_gt(df64 a, df64 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ df64 df_sqr(df64 a) { return df_mul(a, a); }

__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }
__host__ __device__ __forceinline__ df64 df_from_double(double x) {
    float hi = (float)x;
    float lo = (float)(x - (double)hi);
    df64 r;
    r.hi = hi;
    r.lo = lo;
    return r;
}

// ---------------------------------------------------------------- value-type traits
// V   : storage / arithmetic type of ranks and contributions
// Acc : type of the norm / dangling accumulators (FP64-class for every V)
template <typename V> struct Num;

template <> struct Num<double> {
    using V = double;
    using Acc = double;
    __device__ static V zero() { return 0.0; }
    __device__ static V add(V a, V b) { return a + b; }
    __device__ static V add_pos(V a, V b) { return a + b; }
    __device__ static V sub(V a, V b) { return a - b; }
    __device__ static V axpy(V alpha, V x, V c) { return __fma_rn(alpha, x, c); }   // c + alpha*x
    __device__ static V div_int(V x, int32_t d) { return __ddiv_rn(x, (double)d); }
    __device__ static V shfl_xor(V x, int m) { return __shfl_xor_sync(0xffffffffu, x, m); }
    __device__ static double to_double(V x) { return x; }
    __device__ static V from_double(double x) { return x; }
    // accumulator ops
    __device__ static Acc acc_zero() { return 0.0; }
    __device__ static Acc acc_of(V x) { return x; }
    __device__ static Acc acc_add(Acc a, Acc b) { return a + b; }
    __device__ static Acc acc_abs(V d) { return fabs(d); }
    __device__ static Acc acc_sqr(Acc a) { return a * a; }
    __device__ static Acc acc_max(Acc a, Acc b) { return fmax(a, b); }
    __device__ static double acc_to_double(Acc a) { return a; }
    __device__ static Acc acc_shfl_xor(Acc x, int m) { return __shfl_xor_sync(0xffffffffu, x, m); }
};

template <> struct Num<float> {
    using V = float;
    using Acc = df64;
    __device__ static V zero() { return 0.0f; }
    __device__ static V add(V a, V b) { return a + b; }
    __device__ static V add_pos(V a, V b) { return a + b; }
    __device__ static V sub(V a, V b) { return a - b; }
    __device__ static V axpy(V alpha, V x, V c) { return __fmaf_rn(alpha, x, c); }
    __device__ static V div_int(V x, int32_t d) { return __fdiv_rn(x, __int2float_rn(d)); }
    __device__ static V shfl_xor(V x, int m) { return __shfl_xor_sync(0xffffffffu, x, m); }
    __device__ static double to_double(V x) { return (double)x; }
    __device__ static V from_double(double x) { return (float)x; }
    __device__ static Acc acc_zero() { return {0.0f, 0.0f}; }
    __device__ static Acc acc_of(V x) { return {x, 0.0f}; }
    __device__ static Acc acc_add(Acc a, Acc b) { return df_add_pos(a, b); }
    __device__ static Acc acc_abs(V d) { return {fabsf(d), 0.0f}; }
    __device__ static Acc acc_sqr(Acc a) { return df_sqr(a); }
    __device__ static Acc acc_max(Acc a, Acc b) { return df_gt(a, b) ? a : b; }
    __device__ static double acc_to_double(Acc a) { return df_to_double(a); }
    __device__ static Acc acc_shfl_xor(Acc x, int m) {
        return {__shfl_xor_sync(0xffffffffu, x.hi, m), __shfl_xor_sync(0xffffffffu, x.lo, m)};
    }
};

template <> struct Num<df64> {
    using V = df64;
    using Acc = df64;
    __device__ static V zero() { return {0.0f, 0.0f}; }
    __device__ static V add(V a, V b) { return df_add(a, b); }
    __device__ static V add_pos(V a, V b) { return df_add_pos(a, b); }
    __device__ static V sub(V a, V b) { return df_sub(a, b); }
    __device__ static V axpy(V alpha, V x, V c) { return df_add(c, df_mul(alpha, x)); }
    __device__ static V div_int(V x, int32_t d) { return df_div_int(x, d); }
    __device__ static V shfl_xor(V x, int m) {
        return {__shfl_xor_sync(0xffffffffu, x.hi, m), __shfl_xor_sync(0xffffffffu, x.lo, m)};
    }
    __device__ static double to_double(V x) { return df_to_double(x); }
    __device__ static V from_double(double x) { return df_from_double(x); }
    __device__ static Acc acc_zero() { return {0.0f, 0.0f}; }
    __device__ static Acc acc_of(V x) { return x; }
    __device__ static Acc acc_add(Acc a, Acc b) { return df_add_pos(a, b); }
    __device__ static Acc acc_abs(V d) { return df_abs(d); }
    __device__ static Acc acc_sqr(Acc a) { return df_sqr(a); }
    __device__ static Acc acc_max(Acc a, Acc b) { return df_gt(a, b) ? a : b; }
    __device__ static double acc_to_double(Acc a) { return df_to_double(a); }
    __device__ static Acc acc_shfl_xor(Acc x, int m) { return shfl_xor(x, m); }
};

// Per-edge accumulation of non-negative contributions. For df64 the running
// sum keeps the high word with TwoSum and folds every rounding error and low
// word into a separate float (8 FP32 operations per edge); normalise() gives
// a proper double-float at the end of the row.
template <typename V> struct EdgeSum {
    V s;
    __device__ void init() { s = Num<V>::zero(); }
    __device__ void add(V x) { s = Num<V>::add_pos(s, x); }
    __device__ V get() const { return s; }
    __device__ void merge(const EdgeSum &o) { s = Num<V>::add_pos(s, o.s); }
};
template <> struct EdgeSum<df64> {
    float hi, lo;
    __device__ void init() { hi = 0.0f; lo = 0.0f; }
    __device__ void add(df64 x) {
        df64 t = ef_two_sum(hi, x.hi);
        hi = t.hi;
        lo = __fadd_rn(lo, __fadd_rn(t.lo, x.lo));
    }
    __device__ df64 get() const { return ef_fast_two_sum(hi, lo); }
};
