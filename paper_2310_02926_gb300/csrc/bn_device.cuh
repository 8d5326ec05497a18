// bn_device.cuh -- device-side building blocks shared by the particle-pass
// kernels: vector column loads, the exact mesh locator, and the shared-
// memory mesh (count, sums, min, max of a range of bins).
#pragma once

#include <cuda_runtime.h>

#include <climits>

#include "bn_internal.cuh"

namespace bn {

template <typename T> struct VecOf;
template <> struct VecOf<float> { using type = float4; static constexpr int N = 4; };
template <> struct VecOf<double> { using type = double2; static constexpr int N = 2; };

template <typename T>
__device__ __forceinline__ T vget(const typename VecOf<T>::type& v, int j);
template <> __device__ __forceinline__ float vget<float>(const float4& v, int j) {
    return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}
template <> __device__ __forceinline__ double vget<double>(const double2& v, int j) {
    return j == 0 ? v.x : v.y;
}

// Streaming 16-byte column load: evict-first (.cs, the data is read once)
// with a 256-byte L2 prefetch, so the L2 fetches whole line pairs of the
// column from DRAM instead of the sectors one warp asked for.
__device__ __forceinline__ double2 ld_stream(const double2* p) {
    double2 v;
    asm("ld.global.cs.L2::256B.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ float4 ld_stream(const float4* p) {
    float4 v;
    asm("ld.global.cs.L2::256B.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// Mesh location of a particle, -1 when outside.
template <typename T> struct Binner;
template <> struct Binner<float> {
    Axis<float> ax, ay;
    int rx;
    __device__ void init(const GridDesc& g) {
        ax = make_axis<float>(g.ax[0]);
        ay = make_axis<float>(g.ax[1]);
        rx = g.ax[0].res;
    }
    __device__ __forceinline__ int bin(float x, float y) const {
        int ix = axis_bin(ax, x);
        int iy = axis_bin(ay, y);
        return (ix < 0 || iy < 0) ? -1 : iy * rx + ix;
    }
};
template <> struct Binner<double> {
    AxisF64 ax, ay;
    int rx;
    __device__ void init(const GridDesc& g) {
        ax = make_axis_f64(g.ax[0], g.edges[0]);
        ay = make_axis_f64(g.ax[1], g.edges[1]);
        rx = g.ax[0].res;
    }
    __device__ __forceinline__ int bin(double x, double y) const {
        int ix = axis_bin(ax, x);
        int iy = axis_bin(ay, y);
        return (ix < 0 || iy < 0) ? -1 : iy * rx + ix;
    }
};

// IEEE totalOrder key of a value's bits as a signed integer (-0 < +0):
// non-negative patterns keep their bits, negative ones flip the magnitude.
// key_bits inverts it.
template <typename T> struct KeyOf;
template <> struct KeyOf<float> {
    using K = int;
    using K2 = int2;
    static __device__ __forceinline__ int key(float v) {
        const int b = __float_as_int(v);
        return b >= 0 ? b : (b ^ 0x7fffffff);
    }
    static __device__ __forceinline__ float value(int k) {
        return __int_as_float(k >= 0 ? k : (k ^ 0x7fffffff));
    }
    static constexpr int kPosInf = 0x7f800000;
    static constexpr int kNegInf = (int)(0xff800000u ^ 0x7fffffffu);
};
template <> struct KeyOf<double> {
    using K = long long;
    using K2 = longlong2;
    static __device__ __forceinline__ long long key(double v) {
        const long long b = __double_as_longlong(v);
        return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
    }
    static __device__ __forceinline__ double value(long long k) {
        return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffll));
    }
    static constexpr long long kPosInf = 0x7ff0000000000000ll;
    static constexpr long long kNegInf = (long long)(0xfff0000000000000ull ^ 0x7fffffffffffffffull);
};

// ---------------------------------------------------------------- fixed point
// Shared-memory sums as integers. GB300's FP64 pipe is narrow and an FP64
// add to shared memory is a compare-and-swap loop (measured 145 G adds/s
// over the GPU, against 475 G/s for 64-bit integer adds and 1520 G/s for
// 32-bit ones). A kernel picks, per attribute, a scale 2^F from the largest
// exponent among the first values it reads (scale()); a value v whose
// magnitude lies in the 17 binades below 4x that maximum becomes the
// integer q = trunc(v * 2^F), |q| < 2^62, losing at most 2^-45 of |v| (f32
// values convert exactly, over 39 binades); q goes into a 96-bit
// accumulator: a u64 low word (64-bit integer atomic) and a 32-bit high
// word that takes the rare carry or borrow (add96). Integer addition is
// exact and associative, so the accumulated sum is exact up to those
// conversion losses, in any order. Values outside the range (and NaN,
// +-inf, subnormals) are not converted: the caller adds them in FP64
// elsewhere. fixed_value() turns an accumulator back into FP64.
template <typename T> struct Fixed;

template <> struct Fixed<double> {
    static constexpr int kExpMax = 0x7ff;  // inf / NaN
    static constexpr int kDefault = 1023;  // the exponent of 1.0
    static __device__ __forceinline__ int expo(double v) {
        return (int)((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff;
    }
    // The largest sampled biased exponent emax is given two binades of
    // headroom: |v| < 2^(emax - 1021) maps below 2^62.
    static __device__ __forceinline__ int scale(int emax) {
        if (emax <= 0 || emax >= kExpMax) emax = kDefault;
        return 9 + 1075 - (emax + 2);
    }
    // v = +-m * 2^(e - 1075), m the 53-bit significand; q = +-m * 2^sh with
    // sh = e - 1075 + F. Accepted for -7 <= sh <= 9: |q| < 2^62, and at most
    // 7 of m's 53 bits are dropped (relative loss < 2^-45). Zero is q = 0.
    static __device__ __forceinline__ bool to_fixed(double v, int F, long long* q) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        const int e = (int)(b >> 52) & 0x7ff;
        if (e == 0) {
            *q = 0;
            return (b << 1) == 0ull;  // +-0 accepted, subnormals not
        }
        const int sh = e - 1075 + F;
        if (e == kExpMax || sh > 9 || sh < -7) return false;
        const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
        const unsigned long long mag = sh >= 0 ? (m << sh) : (m >> (-sh));
        *q = (b >> 63) ? -(long long)mag : (long long)mag;
        return true;
    }
};

template <> struct Fixed<float> {
    static constexpr int kExpMax = 0xff;
    static constexpr int kDefault = 127;
    static __device__ __forceinline__ int expo(float v) { return (int)(__float_as_uint(v) >> 23) & 0xff; }
    static __device__ __forceinline__ int scale(int emax) {
        if (emax <= 0 || emax >= kExpMax) emax = kDefault;
        return 38 + 150 - (emax + 2);
    }
    // v = +-m * 2^(e - 150), m the 24-bit significand; exact for
    // 0 <= sh = e - 150 + F <= 38 (|q| < 2^62).
    static __device__ __forceinline__ bool to_fixed(float v, int F, long long* q) {
        const unsigned b = __float_as_uint(v);
        const int e = (int)(b >> 23) & 0xff;
        if (e == 0) {
            *q = 0;
            return (b << 1) == 0u;
        }
        const int sh = e - 150 + F;
        if (e == kExpMax || sh > 38 || sh < 0) return false;
        const unsigned long long mag = (unsigned long long)((b & 0x7fffffu) | 0x800000u) << sh;
        *q = (b >> 31) ? -(long long)mag : (long long)mag;
        return true;
    }
};

// 2^k for -1022 <= k <= 1023, from its bits.
__device__ __forceinline__ double pow2(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }

// The signed 96-bit value hi * 2^64 + lo, times 2^-F, as FP64. The scaling
// is two multiplications by powers of two (each factor a normal double for
// |F| <= 2044), exact unless the result falls below the normal range.
__device__ __forceinline__ double fixed_value(unsigned long long lo, int hi, int F) {
    double d;
    if ((hi == 0 && (long long)lo >= 0) || (hi == -1 && (long long)lo < 0))
        d = __ll2double_rn((long long)lo);  // fits in 64 bits: one rounding
    else
        d = __dadd_rn(__dmul_rn((double)hi, 18446744073709551616.0), __ull2double_rn(lo));
    const int f1 = F / 2;
    return __dmul_rn(__dmul_rn(d, pow2(-f1)), pow2(f1 - F));
}


// lo/hi += q as one signed 96-bit integer: a carry out of the low word (q
// >= 0), or an add of a negative q that does not wrap the low word, moves
// the high word.
__device__ __forceinline__ void add96(unsigned long long* lo, int* hi, long long q) {
    const unsigned long long u = (unsigned long long)q;
    const unsigned long long old = atomicAdd(lo, u);
    const bool carry = old + u < old;
    const int d = q >= 0 ? (carry ? 1 : 0) : (carry ? 0 : -1);
    if (d) atomicAdd(hi, d);
}

// Shared-memory mesh of B bins. Sums are FP64 for f64 data and for f32 data
// in kSumF64 mode; FP32 (plus an FP32 compensation term in kSumF32C)
// otherwise. Min and max of one attribute and bin sit next to each other
// as totalOrder keys, so one load reads both and the updates are plain
// signed integer atomicMin / atomicMax.
//
// MODE kSumF64Keys (f64 only): the exact keys are the global key records
// (StateDesc::mmk), and shared memory keeps per bin and attribute the top
// 32 bits of the min and max keys as a filter ([B][A] int2). Every value the
// filter holds belongs to a key already merged into the records, so a
// particle the filter rejects cannot change them; one that passes updates
// the record with a global atomic (an L2 reduction) and lowers (raises) the
// filter. Half the shared-memory bytes per particle for min/max, and the
// mesh leaves more room; data with many values tied at a bin's extreme pays
// one L2 reduction per tied particle instead.
//
// MODE kSumLimbs (f32 only): each sum is an exact integer in three 32-bit
// limbs ([A][3][B]), updated with native 32-bit integer atomics only (on
// GB300 FP32 and 64-bit shared-memory adds are emulated, and on one hot bin
// they fall to a few percent of the integer rate). Per attribute the mesh
// takes a window of 24 binades whose top lies two binades above the largest
// exponent in a sample of the values it will see (sample(), before the
// first add); a value v = +-m 2^(e-150) in the window is the integer
// q = +-m 2^sh, sh = e + 23 - top in [0, 23], so |q| < 2^47 and q = d0 +
// d1 2^16 + d2 2^32 with 16-bit digits d0, d1 >= 0 and a signed d2; the
// limbs add up the digits (zero digits are skipped). With at most
// kLimbMaxAdds values per bin the limbs cannot overflow, and the bin's sum
// is exact until it is rounded once to FP64 in the merge. A value outside
// the window (or 0 < |v| < 2^-126, inf, NaN) is added to the global FP64
// sum directly.
template <typename T, int MODE>
struct SmemMesh {
    static constexpr bool kWide = sizeof(T) == 8 || MODE == kSumF64 || MODE == kSumF64Keys;
    static constexpr bool kGK = MODE == kSumF64Keys;
    static constexpr bool kLimbs = MODE == kSumLimbs;
    static_assert(!kLimbs || sizeof(T) == 4, "limb sums take f32 values");
    using KO = KeyOf<T>;
    using K = typename KO::K;
    using K2 = typename KO::K2;
    unsigned int* cnt;
    double* s64;
    float* s32;
    float* c32;
    K2* mm;  // [A][B] {min key, max key}
    int2* flt;  // kGK: [B][A] {top 32 bits of min key, of max key}
    K2* gkeys;  // kGK: the global key records, gk_rp pairs per bin
    unsigned* lb;          // kLimbs: [A][3][B] digit sums (limb 2 signed)
    int* lexp;             // kLimbs: [A] largest sampled biased exponent
    int* lfb;              // kLimbs: set once a value went to the FP64 sums
    double* const* fsum;   // kLimbs: the global FP64 sums (StateDesc::sum)
    int64_t fbase;         // kLimbs: global bin of local bin 0
    int gk_rp, n_a;
    int B;
    bool do_sum, do_mm, do_min, do_max;

    // kLimbs: where values outside the window go (the global sums of the
    // bins this mesh covers, local bin l being global bin base + l).
    __device__ void bind_fallback(double* const* sums, int64_t base) {
        fsum = sums;
        fbase = base;
    }

    // kLimbs: let value v of attribute a into the sample that sets the
    // window (any thread, between clear() and the barrier before the first
    // add; values of other modes are ignored).
    __device__ __forceinline__ void sample(int a, T v) {
        if constexpr (kLimbs) {
            const int e = (int)(__float_as_uint(v) >> 23) & 0xff;
            if (e > 0 && e < 0xff) atomicMax(&lexp[a], e);
        }
    }

    // kLimbs: the window's top exponent (two binades above the sampled
    // maximum; that of 4.0 with no sample).
    __device__ __forceinline__ int limb_top(int a) const {
        const int e = lexp[a];
        return (e > 0 ? e : 127) + 2;
    }

    // kLimbs: the exact sum of local bin b's limbs, rounded once to FP64.
    __device__ __forceinline__ double limb_value(int a, int b) const {
        const unsigned* L = lb + (size_t)a * 3 * B + b;
        const double hi = (double)(int)L[2 * B] * 4294967296.0;
        const double lo = (double)((unsigned long long)L[B] * 65536ull + L[0]);
        return __dmul_rn(__dadd_rn(hi, lo), pow2(limb_top(a) - 173));
    }

    __device__ void bind_keys(const StateDesc& st) {
        gkeys = static_cast<K2*>(st.mmk);
        gk_rp = key_record_pairs(st.n_attrs, (int)sizeof(K));
    }

    __device__ void carve(unsigned char* base, int B_, int A, bool s, bool lo, bool hi) {
        B = B_;
        do_sum = s;
        do_min = lo;
        do_max = hi;
        do_mm = lo || hi;
        size_t off = ((size_t)B * 4 + 15) & ~(size_t)15;
        cnt = reinterpret_cast<unsigned int*>(base);
        s64 = nullptr;
        s32 = nullptr;
        c32 = nullptr;
        lb = nullptr;
        lexp = nullptr;
        lfb = nullptr;
        fsum = nullptr;
        fbase = 0;
        if (do_sum && kLimbs) {
            lb = reinterpret_cast<unsigned*>(base + off);
            off += (size_t)A * 3 * B * 4;
        } else if (do_sum) {
            if (kWide) {
                s64 = reinterpret_cast<double*>(base + off);
                off += (size_t)A * B * 8;
            } else {
                s32 = reinterpret_cast<float*>(base + off);
                off += (size_t)A * B * 4;
                if (MODE == kSumF32C) {
                    c32 = reinterpret_cast<float*>(base + off);
                    off += (size_t)A * B * 4;
                }
            }
        }
        off = (off + 15) & ~(size_t)15;
        n_a = A;
        mm = (do_mm && !kGK) ? reinterpret_cast<K2*>(base + off) : nullptr;
        flt = (do_mm && kGK) ? reinterpret_cast<int2*>(base + off) : nullptr;
        if (do_mm) off += (size_t)A * B * (kGK ? 8 : sizeof(K2));
        if (kLimbs) {  // [A] sampled exponents, then the fallback flag
            off = (off + 15) & ~(size_t)15;
            lexp = reinterpret_cast<int*>(base + off);
            lfb = lexp + A;
        }
        gkeys = nullptr;
        gk_rp = 0;
    }

    __device__ void clear(int A) {
        for (int b = threadIdx.x; b < B; b += blockDim.x) cnt[b] = 0u;
        const int AB = A * B;
        if (kLimbs) {
            if (do_sum)
                for (int k = threadIdx.x; k < 3 * AB; k += blockDim.x) lb[k] = 0u;
            for (int k = threadIdx.x; k <= A; k += blockDim.x) lexp[k] = 0;  // and the flag
        } else if (do_sum) {
            if (kWide) {
                for (int k = threadIdx.x; k < AB; k += blockDim.x) s64[k] = 0.0;
            } else {
                for (int k = threadIdx.x; k < AB; k += blockDim.x) s32[k] = 0.0f;
                if (MODE == kSumF32C)
                    for (int k = threadIdx.x; k < AB; k += blockDim.x) c32[k] = 0.0f;
            }
        }
        if (do_mm && !kGK) {
            K2 init;
            init.x = KO::kPosInf;
            init.y = KO::kNegInf;
            for (int k = threadIdx.x; k < AB; k += blockDim.x) mm[k] = init;
        }
        if (do_mm && kGK)
            for (int k = threadIdx.x; k < AB; k += blockDim.x) flt[k] = make_int2(INT_MAX, INT_MIN);
    }

    __device__ __forceinline__ void add_count(int b) { atomicAdd(&cnt[b], 1u); }

    __device__ __forceinline__ void add(int a, int b, T v) {
        const int k = a * B + b;
        if (do_sum && kLimbs) {
            const unsigned u = __float_as_uint((float)v);
            const int e = (int)(u >> 23) & 0xff;
            const int sh = e + 23 - limb_top(a);
            if (e > 0 && e < 0xff && sh >= 0 && sh <= 23) {
                const unsigned long long mag = (unsigned long long)((u & 0x7fffffu) | 0x800000u) << sh;
                const long long q = (u >> 31) ? -(long long)mag : (long long)mag;
                const unsigned d0 = (unsigned)q & 0xffffu, d1 = (unsigned)q >> 16;
                const int d2 = (int)(q >> 32);
                unsigned* L = lb + (size_t)a * 3 * B + b;
                if (d0) atomicAdd(L, d0);
                if (d1) atomicAdd(L + B, d1);
                if (d2) atomicAdd(reinterpret_cast<int*>(L + 2 * B), d2);
            } else if ((u << 1) != 0u) {  // +-0 adds nothing
                atomicAdd(fsum[a] + fbase + b, (double)v);
                *lfb = 1;
            }
        } else if (do_sum) {
            if (kWide) {
                atomicAdd(&s64[k], (double)v);
            } else if (MODE == kSumF32) {
                atomicAdd(&s32[k], (float)v);
            } else {
                // Two-sum of the value the atomic added to: the exact rounding
                // error of old + v goes into the compensation term.
                float fv = (float)v;
                float old = atomicAdd(&s32[k], fv);
                float s = __fadd_rn(old, fv);
                float bp = __fsub_rn(s, old);
                float err = __fadd_rn(__fsub_rn(old, __fsub_rn(s, bp)), __fsub_rn(fv, bp));
                // once the sum is +/-inf or NaN the error term is meaningless
                // (inf - inf); the sum itself already carries the result
                if (err != 0.0f && (__float_as_uint(err) & 0x7f800000u) != 0x7f800000u)
                    atomicAdd(&c32[k], err);
            }
        }
        if (do_mm && !kGK) {
            if (is_nan_bits(v)) return;
            const K key = KO::key(v);
            const K2 cur = mm[k];
            if (do_min && key < cur.x) atomicMin(&mm[k].x, key);
            if (do_max && key > cur.y) atomicMax(&mm[k].y, key);
        }
        if (do_mm && kGK) {
            if (is_nan_bits(v)) return;
            const K key = KO::key(v);
            const int h = (int)((long long)key >> 32);  // order preserving
            int2* fp = flt + b * n_a + a;
            const int2 f = *fp;
            K2* kr = gkeys + (int64_t)b * gk_rp + a;
            if (do_min && h <= f.x) {
                atomicMin(&kr->x, key);
                if (h < f.x) atomicMin(&fp->x, h);
            }
            if (do_max && h >= f.y) {
                atomicMax(&kr->y, key);
                if (h > f.y) atomicMax(&fp->y, h);
            }
        }
    }

    // One particle's count and all AC attributes (AC == the mesh's attribute
    // count). Key modes read every attribute's filter pair first, so the
    // loads are in flight while the count and the sums update: 16-byte loads
    // when AC is even (bin b's pairs start at 8 * AC * b bytes, a multiple of
    // 16 only for even AC), 8-byte loads otherwise.
    template <int AC>
    __device__ __forceinline__ void add_particle(int b, const T* v) {
        if constexpr (kGK && AC > 0) {
            int2 f[AC];
            int2* fp = flt + b * AC;
            if (do_mm) {
                if constexpr (AC % 2 == 0) {
#pragma unroll
                    for (int c = 0; c < AC; c += 2) {
                        const int4 q = *reinterpret_cast<const int4*>(fp + c);
                        f[c] = make_int2(q.x, q.y);
                        f[c + 1] = make_int2(q.z, q.w);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < AC; ++c) f[c] = fp[c];
                }
            }
            add_count(b);
            if (do_sum)
#pragma unroll
                for (int a = 0; a < AC; ++a) atomicAdd(&s64[a * B + b], (double)v[a]);
            if (!do_mm) return;
#pragma unroll
            for (int a = 0; a < AC; ++a) {
                if (is_nan_bits(v[a])) continue;
                const K key = KO::key(v[a]);
                const int h = (int)((long long)key >> 32);  // order preserving
                K2* kr = gkeys + (int64_t)b * gk_rp + a;
                if (do_min && h <= f[a].x) {
                    atomicMin(&kr->x, key);
                    if (h < f[a].x) atomicMin(&fp[a].x, h);
                }
                if (do_max && h >= f[a].y) {
                    atomicMax(&kr->y, key);
                    if (h > f[a].y) atomicMax(&fp[a].y, h);
                }
            }
        } else {
            add_count(b);
#pragma unroll
            for (int a = 0; a < AC; ++a) add(a, b, v[a]);
        }
    }

    // Sum of one bin as FP64: the FP64 accumulator, the FP32 partial, or the
    // FP32 partial plus its compensation term (unless the partial is inf/NaN).
    __device__ __forceinline__ double sum_value(int k) const {
        if (kLimbs) return limb_value(k / B, k % B);
        if (kWide) return s64[k];
        if (MODE == kSumF32) return (double)s32[k];
        const float hi = s32[k];
        return ((__float_as_uint(hi) & 0x7f800000u) == 0x7f800000u)
                   ? (double)hi
                   : __dadd_rn((double)hi, (double)c32[k]);
    }

    // CTA partial -> global mesh. Local bin l is global bin base + l; only
    // l < nbins exist. sole: this CTA holds the complete result of these
    // bins, so plain stores replace the atomics (empty bins included);
    // otherwise only non-empty bins are merged.
    __device__ void merge(const StateDesc& st, int A, int64_t base = 0, int nbins = -1,
                          bool sole = false) {
        const int nb = nbins < 0 ? B : nbins;
        for (int l = threadIdx.x; l < nb; l += blockDim.x) {
            const unsigned int c = cnt[l];
            const int64_t b = base + l;
            if (sole) {
                st.count[b] = (unsigned long long)c;
                for (int a = 0; a < A; ++a) {
                    const int k = a * B + l;
                    if (do_sum) {
                        if (kLimbs) {
                            // the global sum holds the values that went
                            // around the limbs (zero when none did)
                            double v = c ? limb_value(a, l) : 0.0;
                            if (c && *lfb) v = __dadd_rn(v, __ldcg(&st.sum[a][b]));
                            st.sum[a][b] = v;
                        } else {
                            st.sum[a][b] = sum_value(k);
                        }
                    }
                    if (do_mm && !kGK) {
                        const K2 cur = mm[k];
                        if (st.mmk) {
                            static_cast<K2*>(st.mmk)[b * key_record_pairs(st.n_attrs, (int)sizeof(K)) + a] = cur;
                        } else {
                            if (do_min) static_cast<T*>(st.mn[a])[b] = KO::value(cur.x);
                            if (do_max) static_cast<T*>(st.mx[a])[b] = KO::value(cur.y);
                        }
                    }
                }
                continue;
            }
            if (c == 0u) continue;
            atomicAdd(&st.count[b], (unsigned long long)c);
            for (int a = 0; a < A; ++a) {
                const int k = a * B + l;
                if (do_sum) atomicAdd(&st.sum[a][b], kLimbs ? limb_value(a, l) : sum_value(k));
                if (kGK) continue;  // min/max already in the global key records
                if (do_mm && st.mmk) {
                    const K2 cur = mm[k];
                    K2* kp = static_cast<K2*>(st.mmk) + b * key_record_pairs(st.n_attrs, (int)sizeof(K)) + a;
                    const K2 g = __ldca(kp);
                    if (do_min && cur.x < g.x) atomicMin(&kp->x, cur.x);
                    if (do_max && cur.y > g.y) atomicMax(&kp->y, cur.y);
                } else if (do_mm) {
                    const K2 cur = mm[k];
                    if (do_min) {
                        const T m = KO::value(cur.x);
                        T* g = static_cast<T*>(st.mn[a]) + b;
                        if (total_less(m, __ldcg(g))) atomic_min_total(g, m);
                    }
                    if (do_max) {
                        const T m = KO::value(cur.y);
                        T* g = static_cast<T*>(st.mx[a]) + b;
                        if (total_less(__ldcg(g), m)) atomic_max_total(g, m);
                    }
                }
            }
        }
    }
};

// Current min/max of a bin for the read-before-atomic filter, through L1.
// L1 is not coherent with the atomics in L2, so the value may be stale; a
// stale min is never below the true min (mins only fall), and a stale max
// never above the true max, so a stale read only admits extra atomics.
template <typename T>
__device__ __forceinline__ T filter_load(const T* p) { return __ldca(p); }

// The first np pairs (a multiple of the pairs in 32 bytes) of bin b's key
// record (StateDesc::mmk), read with 256-bit loads: one L2 request per two
// f64 (four f32) attributes. Cached in L1 like filter_load: a stale record
// only lets through an atomic that turns out to be unnecessary.
__device__ __forceinline__ void load_key_record(const longlong2* rec, longlong2* out, int np) {
    if (np == 1) {  // a 16-byte record
        out[0] = __ldca(rec);
        return;
    }
    for (int c = 0; c < np; c += 2) {
        unsigned long long w0, w1, w2, w3;
        asm("ld.global.ca.v4.u64 {%0, %1, %2, %3}, [%4];"
            : "=l"(w0), "=l"(w1), "=l"(w2), "=l"(w3)
            : "l"(rec + c));
        out[c] = make_longlong2((long long)w0, (long long)w1);
        out[c + 1] = make_longlong2((long long)w2, (long long)w3);
    }
}
__device__ __forceinline__ void load_key_record(const int2* rec, int2* out, int np) {
    if (np == 2) {  // a 16-byte record
        const int4 v = __ldca(reinterpret_cast<const int4*>(rec));
        out[0] = make_int2(v.x, v.y);
        out[1] = make_int2(v.z, v.w);
        return;
    }
    for (int c = 0; c < np; c += 4) {
        unsigned long long w[4];
        asm("ld.global.ca.v4.u64 {%0, %1, %2, %3}, [%4];"
            : "=l"(w[0]), "=l"(w[1]), "=l"(w[2]), "=l"(w[3])
            : "l"(rec + c));
#pragma unroll
        for (int j = 0; j < 4; ++j)
            out[c + j] = make_int2((int)(unsigned)(w[j] & 0xffffffffu), (int)(unsigned)(w[j] >> 32));
    }
}

// Key pairs of a record / filter pairs of a filter record that a compile-time
// attribute count needs in registers (kMaxAttr when the count is not fixed).
template <typename K2, int A_CT>
struct RecPairs {
    static constexpr int Q = 32 / (int)sizeof(K2);
    static constexpr int value = A_CT > 0 ? (A_CT + Q - 1) / Q * Q : kMaxAttr;
};
template <int A_CT>
struct FltPairs {
    static constexpr int value = A_CT > 0 ? (A_CT + 3) / 4 * 4 : kMaxAttr;
};

// Min and max of one particle (lo == hi == its values), or of a combined
// group of particles (lo / hi: the group's min / max per attribute, +inf /
// -inf where the group has no non-NaN value), into bin b's state. Three
// forms of the state:
//  - f64 key records behind the 32-bit filter (st.mmf): one 256-bit filter
//    read per four attributes; only a key whose top half reaches the
//    filter's bound updates the record, then lowers (raises) the filter;
//  - key records alone (st.mmk): the record is read, an atomic is issued
//    only where the key would change it;
//  - the outputs themselves (raw IEEE bits, totalOrder atomics).
// The f64 filter form of commit_minmax once bin b's filter record f has been
// read (load_filter): only keys whose top half reaches the filter's bound
// update the key record, then lower (raise) the filter.
template <int A_CT>
__device__ __forceinline__ void apply_filtered_minmax(const StateDesc& st, int A, int64_t b, const double* lo,
                                                      const double* hi, const int2* f) {
    using KO = KeyOf<double>;
    using K2 = typename KO::K2;
    int2* fr = static_cast<int2*>(st.mmf) + b * filter_record_pairs(st.n_attrs);
    K2* kr = static_cast<K2*>(st.mmk) + b * key_record_pairs(st.n_attrs, (int)sizeof(typename KO::K));
    for (int a = 0; a < A; ++a) {
        const long long kl = KO::key(lo[a]), kh = KO::key(hi[a]);
        const int hl = (int)(kl >> 32), hh = (int)(kh >> 32);  // order preserving
        if (st.do_min && hl <= f[a].x && !is_nan_bits(lo[a])) {
            atomicMin(&kr[a].x, kl);
            if (hl < f[a].x) atomicMin(&fr[a].x, hl);
        }
        if (st.do_max && hh >= f[a].y && !is_nan_bits(hi[a])) {
            atomicMax(&kr[a].y, kh);
            if (hh > f[a].y) atomicMax(&fr[a].y, hh);
        }
    }
}

// Bin b's f64 filter record (st.mmf set), FltPairs<A_CT> pairs.
template <int A_CT>
__device__ __forceinline__ void load_filter(const StateDesc& st, int A, int64_t b, int2* f) {
    const int2* fr = static_cast<const int2*>(st.mmf) + b * filter_record_pairs(st.n_attrs);
    load_key_record(fr, f, filter_record_pairs(A));
}

template <typename T, int A_CT>
__device__ __forceinline__ void commit_minmax(const StateDesc& st, int A, int64_t b, const T* lo,
                                              const T* hi) {
    if (!(st.do_min || st.do_max)) return;
    using KO = KeyOf<T>;
    using K2 = typename KO::K2;
    if constexpr (sizeof(T) == 8) {
        if (st.mmf) {
            int2 f[FltPairs<A_CT>::value];
            load_filter<A_CT>(st, A, b, f);
            apply_filtered_minmax<A_CT>(st, A, b, lo, hi, f);
            return;
        }
    }
    if (st.mmk) {
        constexpr int RP = RecPairs<K2, A_CT>::value;
        K2 rec[RP];
        K2* kr = static_cast<K2*>(st.mmk) + b * key_record_pairs(st.n_attrs, (int)sizeof(typename KO::K));
        load_key_record(kr, rec, key_record_pairs(A, (int)sizeof(typename KO::K)));
        for (int a = 0; a < A; ++a) {
            if (st.do_min && !is_nan_bits(lo[a])) {
                const auto kl = KO::key(lo[a]);
                if (kl < rec[a].x) atomicMin(&kr[a].x, kl);
            }
            if (st.do_max && !is_nan_bits(hi[a])) {
                const auto kh = KO::key(hi[a]);
                if (kh > rec[a].y) atomicMax(&kr[a].y, kh);
            }
        }
        return;
    }
    for (int a = 0; a < A; ++a) {
        if (st.do_min && !is_nan_bits(lo[a])) {
            T* g = static_cast<T*>(st.mn[a]) + b;
            if (total_less(lo[a], filter_load(g))) atomic_min_total(g, lo[a]);
        }
        if (st.do_max && !is_nan_bits(hi[a])) {
            T* g = static_cast<T*>(st.mx[a]) + b;
            if (total_less(filter_load(g), hi[a])) atomic_max_total(g, hi[a]);
        }
    }
}

// A value the bulk record reduction carries: zero or a normal finite
// double. Subnormal, infinite and NaN values go to the record's element
// through a plain FP64 reduction instead, so they behave exactly as on every
// other path. Integer tests on the bits (no FP64 compare).
__device__ __forceinline__ bool record_plain(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned e = (unsigned)(u >> 52) & 0x7ffu;
    return (e - 1u) < 0x7feu || (u << 1) == 0ull;
}

// Bulk reduction of a staged record: the copy engine adds the RD doubles of
// this thread's shared-memory slot (16-byte aligned) element-wise into dst
// (16-byte aligned, RD even) in L2, as one operation. record_slot_ready()
// must come before the slot is written: it returns once the thread's
// previous reduction has read the slot.
__device__ __forceinline__ void record_slot_ready() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
template <int RD>
__device__ __forceinline__ void record_reduce(double* dst, const double* slot) {
    static_assert(RD % 2 == 0, "records are whole 16-byte pieces");
    // the generic-proxy stores must be visible to the async proxy's read
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;"
                 :: "l"(dst), "r"((unsigned)__cvta_generic_to_shared(slot)), "n"(RD * 8)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until every bulk reduction this thread issued has completed (before
// the thread exits: its slot lives in the CTA's shared memory).
__device__ __forceinline__ void record_drain() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Count cnt and the FP64 sums s of bin b: one bulk reduction of the bin's
// count-and-sums record when the caller passes a slot (st.rec set, the
// attribute count known at compile time), else 1 + A reductions.
template <int A_CT>
__device__ __forceinline__ void commit_count_sums(const StateDesc& st, int A, int b, unsigned long long cnt,
                                                  const double* s, double* slot) {
    if constexpr (A_CT >= 1) {
        if (slot) {
            constexpr int RD = (A_CT + 2) & ~1;
            double* dst = st.rec + (int64_t)b * RD;
            // element k of the record: the count (exact: cnt <= 32), a plain
            // sum, or 0.0 (padding, and sums that take the FP64 reduction)
            auto elem = [&](int k) -> double {
                if (k == 0) return (double)cnt;
                if (k > A_CT) return 0.0;
                return record_plain(s[k - 1]) ? s[k - 1] : 0.0;
            };
#pragma unroll
            for (int a = 0; a < A_CT; ++a)
                if (!record_plain(s[a])) atomicAdd(dst + 1 + a, s[a]);
            record_slot_ready();
#pragma unroll
            for (int k = 0; k < RD; k += 2)
                *reinterpret_cast<double2*>(slot + k) = make_double2(elem(k), elem(k + 1));
            record_reduce<RD>(dst, slot);
            return;
        }
    }
    atomicAdd(&st.count[b], cnt);
    if (st.do_sum)
        for (int a = 0; a < A; ++a) atomicAdd(&st.sum[a][b], s[a]);
}

// Combine the lanes of the calling warp that share bin b (b >= 0) and let
// the lowest such lane update the global mesh. Every lane of the warp must
// call it (b = -1 for lanes without an in-bounds particle). slot: this
// thread's record staging slot when the count and sums go out as records
// (st.rec), else null.
template <typename T, int A_CT>
__device__ __forceinline__ void warp_commit(const StateDesc& st, int A, int b, const T* v,
                                            bool aggregate, double* slot = nullptr) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned peers = aggregate ? __match_any_sync(full, b) : (1u << lane);
    const int leader = __ffs(peers) - 1;
    const bool alone = peers == (1u << lane);
    if (!aggregate || __all_sync(full, alone || b < 0)) {
        // no two lanes share a bin: skip the combining shuffles
        if (b < 0) return;
        if constexpr (A_CT >= 1) {
            if (slot) {  // (a record slot implies sums)
                double vs[A_CT];
#pragma unroll
                for (int a = 0; a < A_CT; ++a) vs[a] = (double)v[a];
                commit_count_sums<A_CT>(st, A, b, 1ull, vs, slot);
                commit_minmax<T, A_CT>(st, A, b, v, v);
                return;
            }
        }
        atomicAdd(&st.count[b], 1ull);
        if (st.do_sum)
            for (int a = 0; a < A; ++a) atomicAdd(&st.sum[a][b], (double)v[a]);
        commit_minmax<T, A_CT>(st, A, b, v, v);
        return;
    }
    // General case: the leader of each peer group gathers its peers' values
    // lane by lane (the loop runs over the largest group in the warp).
    const unsigned cnt = __popc(peers);
    double s[A_CT > 0 ? A_CT : kMaxAttr];
    T lo[A_CT > 0 ? A_CT : kMaxAttr], hi[A_CT > 0 ? A_CT : kMaxAttr];
    for (int a = 0; a < A; ++a) {
        s[a] = 0.0;
        lo[a] = pos_inf<T>();
        hi[a] = neg_inf<T>();
    }
    unsigned rest = peers;
    // every lane walks its own group; shuffles need all lanes, so loop to the
    // warp-wide maximum group size
    int my_n = (b >= 0) ? (int)cnt : 0;
    int max_n = my_n;
    for (int off = 16; off > 0; off >>= 1) max_n = max(max_n, __shfl_xor_sync(full, max_n, off));
    for (int it = 0; it < max_n; ++it) {
        int src = rest ? __ffs(rest) - 1 : lane;
        if (rest) rest &= rest - 1;
        for (int a = 0; a < A; ++a) {
            T x = __shfl_sync(full, v[a], src);
            if (b >= 0 && it < my_n) {
                s[a] += (double)x;  // FP64 add in this lane's registers
                if (!is_nan_bits(x)) {
                    if (total_less(x, lo[a])) lo[a] = x;
                    if (total_less(hi[a], x)) hi[a] = x;
                }
            }
        }
    }
    if (b < 0 || lane != leader) return;
    commit_count_sums<A_CT>(st, A, b, (unsigned long long)cnt, s, slot);
    // +inf / -inf where the group holds no non-NaN value: an atomic with them
    // changes nothing, and the direct form skips them
    commit_minmax<T, A_CT>(st, A, b, lo, hi);
}

}  // namespace bn
