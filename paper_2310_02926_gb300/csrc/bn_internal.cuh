// bn_internal.cuh -- device helpers and launch descriptors shared by the
// binning kernels (Sec. 4.2 data binning) and the host runtime.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/binning.h"

namespace bn {

constexpr int kMaxAttr = BN_MAX_ATTR;

// ---------------------------------------------------------------- sum modes
// kSumF64Keys: FP64 sums; the exact min/max keys live in global key
// records (StateDesc::mmk) behind a 32-bit filter in shared memory (private
// strategy, f64 data).
// kSumLimbs (f32 data, shared-memory meshes only): exact fixed-point sums in
// three 32-bit integer limbs (see SmemMesh). It serves the kSumF32C and
// kSumF64 requests of shared-memory meshes: on GB300 only 32-bit integer
// shared-memory atomics are native; FP32 and 64-bit adds are emulated and
// slow down sharply when many threads hit one bin.
enum SumMode : int { kSumF32C = 0, kSumF32 = 1, kSumF64 = 2, kSumF64Keys = 3, kSumLimbs = 4 };

// The most values one kSumLimbs mesh may add into one bin between its clear
// and its merge (the headroom of its 16-bit digits in 32-bit limbs).
constexpr int kLimbMaxAdds = 65536;

// The shared-memory mesh mode for a request's sum mode and data type.
__host__ __device__ __forceinline__ int smem_sum_mode(int dtype, int sum_mode) {
    if (dtype == BN_F64) return kSumF64;
    return sum_mode == kSumF32 ? kSumF32 : kSumLimbs;
}

// ---------------------------------------------------------------- mesh axis
// One axis of the mesh with bounds and scale already rounded to the
// coordinate type T (stored widened in double). closed = automatic bounds.
struct AxisDesc {
    double lo, hi, s;
    int32_t res;
    int32_t closed;
    // f64 coordinates only: 1 when the FP32 estimate of t is within `delta`
    // bins of the exact t everywhere on the axis, with delta < 1/4 (then the
    // estimate plus the edge-key correction below is exact); 0 = the
    // estimate only seeds a search of the edge keys.
    int32_t fast;
    float delta;
};

// The mesh as the kernels see it. For explicit bounds the host fills it;
// for automatic bounds the bounds kernel writes it into device memory and
// sets valid (0 = degenerate: the request fails, nothing is binned).
struct GridDesc {
    AxisDesc ax[2];
    int32_t valid;
    int32_t pad;
    // Exact bin-edge keys for f64 coordinates (see EdgeTables): device
    // pointers to res+1 ordered keys per axis, or nullptr.
    const long long* edges[2];
};

// ---------------------------------------------------------------- columns
template <typename T>
struct Columns {
    const T* x;
    const T* y;
    const T* a[kMaxAttr];
    int64_t n;
};

// Per-bin state in global memory; these are the output buffers themselves
// (or library scratch standing in for outputs the caller did not ask for).
struct StateDesc {
    unsigned long long* count;
    double* sum[kMaxAttr];
    void* mn[kMaxAttr];
    void* mx[kMaxAttr];
    double* avg[kMaxAttr];
    // Optional min/max state as totalOrder keys: per bin one record of
    // key_record_pairs(n_attrs, sizeof T) pairs {min key, max key} (long long
    // for f64, int for f32), attribute a at pair a, padded to 16 bytes or to
    // whole 32-byte pieces so that one 256-bit load reads the pairs of two
    // f64 (four f32) attributes. When set, the particle pass updates these instead of mn/mx
    // and k_finalize writes mn/mx from them; when null, mn/mx hold the
    // running min/max directly.
    void* mmk;
    // Optional filter in front of f64 key records (global strategy, three or
    // more attributes): per bin filter_record_pairs(n_attrs) int2 pairs {top
    // 32 bits of the min key, of the max key}, 32 bytes per four attributes,
    // so one 256-bit load tells whether a particle can change any of the
    // record's keys (a key whose top half is above the filter's min cannot
    // lower the min). Only the keys that pass reach the records.
    void* mmf;
    // Optional count-and-sums records (global strategy, 1..kRecMaxAttr
    // attributes with sums): per bin record_doubles(n_attrs) doubles {count,
    // sum of attribute 0, ..., zero padding}, 16-byte aligned, so that one
    // particle's count and sums reach L2 as one bulk reduction of the whole
    // record instead of 1 + n_attrs separate reductions. The count is held
    // as a double: adding 1.0 to an integer-valued double is exact below
    // 2^53. When set, the particle pass updates these instead of count/sum
    // and k_finalize writes count and sum from them.
    double* rec;
    int64_t bins;
    int32_t n_attrs;
    int32_t do_sum;  // sums needed (SUM or AVG requested)
    int32_t do_min;
    int32_t do_max;
    int32_t do_avg;
    int32_t pad;
};

// Attribute counts whose count-and-sums records the global kernel handles.
constexpr int kRecMaxAttr = 4;

// Doubles per count-and-sums record: the count, one sum per attribute,
// rounded up to whole 16-byte pieces (a bulk reduction moves multiples of
// 16 bytes).
__host__ __device__ __forceinline__ int record_doubles(int n_attrs) { return (n_attrs + 2) & ~1; }

// Key pairs per bin record of StateDesc::mmk: a record of at most 16 bytes is
// padded to 16 (one 128-bit load), a longer one to whole 32-byte pieces
// (256-bit loads: 2 pairs of 8-byte keys, 4 of 4-byte keys per piece).
__host__ __device__ __forceinline__ int key_record_pairs(int n_attrs, int key_bytes) {
    const int pair = 2 * key_bytes;
    if (n_attrs * pair <= 16) return 16 / pair;
    const int q = 32 / pair;
    return (n_attrs + q - 1) / q * q;
}

// int2 pairs per bin of StateDesc::mmf: whole 32-byte pieces of four pairs.
__host__ __device__ __forceinline__ int filter_record_pairs(int n_attrs) {
    return (n_attrs + 3) / 4 * 4;
}

// ---------------------------------------------------------------- bits
__device__ __forceinline__ bool is_nan_bits(float v) {
    return (__float_as_uint(v) & 0x7fffffffu) > 0x7f800000u;
}
// The f64 test is spelled in PTX so that it stays two integer instructions:
// written in C, the compiler may turn it into an unordered FP64 compare, which
// runs on GB300's narrow FP64 pipe and, being side-effect free, can be hoisted
// out of the branches that need it into every particle's path.
__device__ __forceinline__ bool is_nan_bits(double v) {
    unsigned int r;
    asm("{\n\t.reg .pred p;\n\t.reg .b64 m;\n\t"
        "and.b64 m, %1, 0x7fffffffffffffff;\n\t"
        "setp.gt.u64 p, m, 0x7ff0000000000000;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "l"(__double_as_longlong(v)));
    return r != 0;
}

// Ordered integer key of an IEEE value: key(a) < key(b) iff a < b for
// non-NaN a, b, with -0 and +0 both mapped to key 0 (they compare equal).
__device__ __forceinline__ long long ordered_key(double v) {
    long long b = __double_as_longlong(v);
    if (b == (long long)0x8000000000000000ull) b = 0;
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}
__device__ __forceinline__ int ordered_key(float v) {
    int b = __float_as_int(v);
    if (b == (int)0x80000000u) b = 0;
    return b >= 0 ? b : (b ^ 0x7fffffff);
}

// ---------------------------------------------------------------- min / max
// IEEE totalOrder min/max through integer atomics on the value's own bits:
// non-negative values (sign bit 0) order like signed integers, negative
// values order reversed like unsigned integers, and every negative bit
// pattern is above every non-negative one as unsigned. So a min with a
// non-negative value is a signed atomicMin and a min with a negative value
// is an unsigned atomicMax (and the mirror image for max). Works in shared
// and global memory; the location must hold a non-NaN value (init +/-inf).
__device__ __forceinline__ void atomic_min_total(float* p, float v) {
    int b = __float_as_int(v);
    if (b >= 0) atomicMin(reinterpret_cast<int*>(p), b);
    else atomicMax(reinterpret_cast<unsigned int*>(p), static_cast<unsigned int>(b));
}
__device__ __forceinline__ void atomic_max_total(float* p, float v) {
    int b = __float_as_int(v);
    if (b >= 0) atomicMax(reinterpret_cast<int*>(p), b);
    else atomicMin(reinterpret_cast<unsigned int*>(p), static_cast<unsigned int>(b));
}
__device__ __forceinline__ void atomic_min_total(double* p, double v) {
    long long b = __double_as_longlong(v);
    if (b >= 0) atomicMin(reinterpret_cast<long long*>(p), b);
    else atomicMax(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(b));
}
__device__ __forceinline__ void atomic_max_total(double* p, double v) {
    long long b = __double_as_longlong(v);
    if (b >= 0) atomicMax(reinterpret_cast<long long*>(p), b);
    else atomicMin(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(b));
}

// totalOrder "a < b" for non-NaN a, b on the value bits (integer pipe only).
__device__ __forceinline__ bool total_less(float a, float b) {
    int ia = __float_as_int(a), ib = __float_as_int(b);
    int ka = ia >= 0 ? ia : (ia ^ 0x7fffffff);
    int kb = ib >= 0 ? ib : (ib ^ 0x7fffffff);
    return ka < kb;
}
__device__ __forceinline__ bool total_less(double a, double b) {
    long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    long long ka = ia >= 0 ? ia : (ia ^ 0x7fffffffffffffffll);
    long long kb = ib >= 0 ? ib : (ib ^ 0x7fffffffffffffffll);
    return ka < kb;
}

template <typename T> __device__ __forceinline__ T pos_inf();
template <> __device__ __forceinline__ float pos_inf<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double pos_inf<double>() {
    return __longlong_as_double(0x7ff0000000000000ll);
}
template <typename T> __device__ __forceinline__ T neg_inf();
template <> __device__ __forceinline__ float neg_inf<float>() { return __int_as_float(0xff800000); }
template <> __device__ __forceinline__ double neg_inf<double>() {
    return __longlong_as_double((long long)0xfff0000000000000ull);
}

// ---------------------------------------------------------------- average
// avg = RN(sum / count) for count >= 1 (Sec. 4.2's per-bin average, in
// FP64). A power-of-two count divides exactly by scaling, so count 1 is the
// sum itself and count 2^k one FP64 multiplication by 2^-k (rounded once,
// as the quotient would be); other counts take the FP64 division, which on
// GB300's narrow FP64 pipe runs at about a quarter of the memory rate
// (measured 58 G divisions/s) and bounds a finalise pass over many
// occupied bins.
__device__ __forceinline__ double bin_average(double sum, unsigned long long count) {
    if ((count & (count - 1)) == 0ull) {
        if (count == 1ull) return sum;
        const int k = 63 - __clzll((long long)count);
        return __dmul_rn(sum, __longlong_as_double((long long)(1023 - k) << 52));
    }
    return __ddiv_rn(sum, (double)count);
}

// ---------------------------------------------------------------- bin index
// Axis in the coordinate's own type, prepared once per thread.
template <typename T>
struct Axis {
    T lo, hi, s;
    int res;
    bool closed;
};

template <typename T>
__device__ __forceinline__ Axis<T> make_axis(const AxisDesc& d) {
    Axis<T> a;
    a.lo = (T)d.lo;
    a.hi = (T)d.hi;
    a.s = (T)d.s;
    a.res = d.res;
    a.closed = d.closed != 0;
    return a;
}

// Nearest integer of t (0 <= t < 2^22) with plain round-to-nearest FP32 adds
// and integer operations only. GB300 runs float-to-integer conversions and
// rounding instructions on its narrow FP64 pipe; here, adding 1.5 * 2^23
// (bits 0x4B400000) lands in [2^23, 2^24) where the ulp is 1, so the sum is
// 1.5 * 2^23 + round(t) exactly and its low bits are round(t). *d receives
// t - round(t), exact (Sterbenz, or t itself when the rounded value is 0),
// with |d| <= 1/2.
__device__ __forceinline__ int round_small(float t, float* d) {
    const float s = __fadd_rn(t, 12582912.0f);
    *d = __fsub_rn(t, __fsub_rn(s, 12582912.0f));
    return __float_as_int(s) - 0x4B400000;
}

// The reference sequence (Sec. 4.2 bin location, rounding fixed as
// t = RN(RN(x - lo) * s), i = min(trunc(t), res - 1)), in f32. Inside the
// mesh t >= 0 (t is -0 only when x = -0 and lo = +0) and t is within a few
// ulps of at most res <= 65536 < 2^22, so trunc(t) = floor(t), taken from
// round_small.
__device__ __forceinline__ int axis_bin(const Axis<float>& a, float x) {
    bool inside = a.closed ? (a.lo <= x && x <= a.hi) : (a.lo <= x && x < a.hi);
    if (!inside) return -1;
    float t = __fmul_rn(__fsub_rn(x, a.lo), a.s);
    float d;
    const int r = round_small(t, &d);
    return min(d < 0.0f ? r - 1 : r, a.res - 1);  // floor; t = -0 gives d = -0, not < 0
}

// Inverse of ordered_key(double).
__host__ __device__ __forceinline__ double key_to_double(long long k) {
    long long b = k >= 0 ? k : (k ^ 0x7fffffffffffffffll);
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b);
#else
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
#endif
}

// FP32 approximation of a double from its top 32 bits, integer pipe only:
// the magnitude is truncated to 20 mantissa bits (relative error < 2^-20);
// |x| < 2^-126 becomes +/-0 and |x| >= 2^128 becomes +/-inf.
// Spelled in PTX for the same reason as is_nan_bits(double): the range tests
// on the high word must not become FP64 compares. Exponent bias change:
// 896 << 20 = 0x38000000; 897 << 20 = 0x38100000; 1151 << 20 = 0x47F00000.
__device__ __forceinline__ float approx_float(double x) {
    unsigned int r;
    asm("{\n\t.reg .b32 lo, hi, mag, sgn, v, w;\n\t.reg .pred p, q;\n\t"
        "mov.b64 {lo, hi}, %1;\n\t"
        "and.b32 mag, hi, 0x7fffffff;\n\t"
        "and.b32 sgn, hi, 0x80000000;\n\t"
        "sub.u32 v, mag, 0x38000000;\n\t"
        "shl.b32 v, v, 3;\n\t"
        "or.b32 v, v, sgn;\n\t"
        "setp.lt.u32 p, mag, 0x38100000;\n\t"
        "selp.b32 v, sgn, v, p;\n\t"
        "setp.ge.u32 q, mag, 0x47F00000;\n\t"
        "or.b32 w, sgn, 0x7f800000;\n\t"
        "selp.b32 %0, w, v, q;\n\t}"
        : "=r"(r)
        : "l"(__double_as_longlong(x)));
    return __uint_as_float(r);
}

// f64 axis for the exact edge-key method. idx(x) = min(trunc(RN(RN(x-lo)*s)),
// res-1) is non-decreasing in x, so bin i is the key interval
// [E[i], E[i+1]) where E[i] is the smallest ordered key whose value has
// idx >= i (E[0] = key(lo); E[res] = key(hi), plus one when closed). The
// kernel estimates i in FP32, then moves it by at most one bin so that
// E[i] <= key(x) < E[i+1]: the same index as the reference sequence, with
// no FP64 arithmetic. Every f64 axis has its edge keys, so this is the only
// per-particle path: when the estimate's error is not proven below 1/4 bin
// (huge coordinates or scales), the estimate only seeds the search. (A
// branch into an FP64 evaluation here would cost every particle: the
// compiler hoists parts of it out of the branch, onto the FP64 pipe.)
struct AxisF64 {
    const long long* E;  // res + 1 edge keys
    long long klo, khi;  // E[0], E[res]
    float flo, fs;       // FP32 estimate parameters
    float delta;         // bound on |estimate - t| in bins; +inf if unproven
    float tmax;          // res - delta
    float tlast;         // res - 1
    int res;
};

__device__ __forceinline__ AxisF64 make_axis_f64(const AxisDesc& d, const long long* E) {
    AxisF64 a;
    a.E = E;
    a.res = d.res;
    a.flo = approx_float(d.lo);
    a.fs = (float)d.s;  // may round to inf when !fast; the search handles it
    a.delta = d.fast ? d.delta : __int_as_float(0x7f800000);
    a.tmax = (float)d.res - a.delta;
    a.tlast = (float)(d.res - 1);
    a.klo = __ldg(E);
    a.khi = __ldg(E + d.res);
    return a;
}

// Exact bin of x on an f64 axis (-1 outside). Fast path: the FP32 estimate
// t_f is within delta of the reference t, so when t_f lies in
// (delta, res - delta) and at least delta away from the nearest integer,
// x is inside and trunc(t) == trunc(t_f). Otherwise (about 2 * delta of the
// particles, every particle outside or near the ends, and every particle of
// an axis without a proven delta) the ordered key of x is compared with the
// exact edge keys, starting from the estimate.
__device__ __forceinline__ int axis_bin(const AxisF64& a, double x) {
    const float t = __fmul_rn(__fsub_rn(approx_float(x), a.flo), a.fs);
    if (t > a.delta && t < a.tmax) {  // then 0 < t < res <= 65536
        // t is more than delta from every integer iff |t - round(t)| > delta
        // (delta < 1/4), and then trunc(t) = floor(t) = round(t) - (d < 0)
        float d;
        const int r = round_small(t, &d);
        if (fabsf(d) > a.delta) return d < 0.0f ? r - 1 : r;
    }
    const long long k = ordered_key(x);
    if (k < a.klo || k >= a.khi) return -1;  // NaN keys fall outside too
    // seed: floor of the estimate clamped to [0, res - 1] (fmaxf maps NaN to 0)
    float d;
    const float tc = fminf(fmaxf(t, 0.0f), a.tlast);
    const int r = round_small(tc, &d);
    int i = d < 0.0f ? r - 1 : r;
    i = max(0, min(i, a.res - 1));
    if (k < __ldg(a.E + i)) {
        i -= 1;
    } else if (k >= __ldg(a.E + i + 1)) {
        i += 1;
    }
    i = max(0, min(i, a.res - 1));
    if (k < __ldg(a.E + i) || k >= __ldg(a.E + i + 1)) {
        // the seed was more than one bin off: binary search, E[lo] <= k < E[hi]
        int lo = 0, hi = a.res;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (k >= __ldg(a.E + mid)) lo = mid; else hi = mid;
        }
        i = lo;
    }
    return i;
}

// ---------------------------------------------------------------- edge keys
// Reference bin index on the FP64 pipe (used only to locate edges).
__device__ __forceinline__ int ref_idx_f64(const AxisDesc& d, double x) {
    double t = __dmul_rn(__dsub_rn(x, d.lo), d.s);
    int k = __double2int_rz(t);
    return min(k, d.res - 1);
}

__device__ __forceinline__ long long key_of(double v) { return ordered_key(v); }

// E[i]: the smallest ordered key whose value has bin index >= i. The index
// is non-decreasing in the key, so a bracketing search finds it; it starts
// at the key of lo + i / s and gallops outwards.
__device__ inline long long edge_key(const AxisDesc& d, int i) {
    const long long K0 = key_of(d.lo);
    const long long Khi = key_of(d.hi) + (d.closed ? 1 : 0);
    if (i <= 0) return K0;
    if (i >= d.res) return Khi;
    // invariant: f(lo_k) false (index < i), f(hi_k) true (index >= i; Khi by
    // convention since hi itself indexes to res - 1 >= i)
    long long lo_k = K0, hi_k = Khi;
    auto f = [&](long long k) { return ref_idx_f64(d, key_to_double(k)) >= i; };
    auto gap = [&]() { return (unsigned long long)hi_k - (unsigned long long)lo_k; };
    if (gap() > 2) {
        double est = __dadd_rn(d.lo, __ddiv_rn((double)i, d.s));
        long long e = key_of(est);
        if (e <= lo_k) e = lo_k + 1;
        if (e >= hi_k) e = hi_k - 1;
        if (f(e)) {
            hi_k = e;
            unsigned long long step = 1;
            for (int it = 0; it < 64 && gap() > 1; ++it) {
                if (step >= gap()) break;
                long long c = hi_k - (long long)step;
                if (f(c)) { hi_k = c; step <<= 1; } else { lo_k = c; break; }
            }
        } else {
            lo_k = e;
            unsigned long long step = 1;
            for (int it = 0; it < 64 && gap() > 1; ++it) {
                if (step >= gap()) break;
                long long c = lo_k + (long long)step;
                if (f(c)) { hi_k = c; break; } else { lo_k = c; step <<= 1; }
            }
        }
    }
    for (int it = 0; it < 70 && gap() > 1; ++it) {
        long long mid = lo_k + (long long)(gap() >> 1);
        if (f(mid)) hi_k = mid; else lo_k = mid;
    }
    return hi_k;
}


// ---------------------------------------------------------------- launch info
struct LaunchCfg {
    int grid;
    int block;
    size_t smem;
};

}  // namespace bn
