// Shared device-side definitions of the stencil engine.
//
// Geometry convention: axis 0 is the slowest axis, axis DIMS-1 the contiguous
// one.  Coordinates inside kernels are STORAGE coordinates: for Dirichlet
// grids the ring of width 1 sits at storage index 0 and n_a + 1, the interior
// at 1..n_a; for periodic grids storage and interior coincide (0..n_a-1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pcot {

constexpr int kMaxDims = 3;

struct DevGeo {
    int64_t e[kMaxDims];  // stored extent per axis
    int64_t s[kMaxDims];  // element stride per axis (s[dims-1] == 1)
    int64_t n[kMaxDims];  // interior size per axis
    int32_t dims;
    int32_t periodic;
};

template <class T>
struct Coeffs {
    T c[7];  // centre, axis0 -1, axis0 +1, axis1 -1, axis1 +1, axis2 -1, axis2 +1
};

// Arithmetic policy of the point update.  EXACT: every multiply and add is
// separately rounded (binary64, round to nearest even) in the coefficient
// order, which reproduces a plain evaluation of the definition bit for bit.
// Otherwise the products are fused into the running sum (fma).
template <class T, bool EXACT>
struct Arith;

template <>
struct Arith<double, true> {
    static __device__ __forceinline__ double first(double c, double u) { return __dmul_rn(c, u); }
    static __device__ __forceinline__ double acc(double a, double c, double u) { return __dadd_rn(a, __dmul_rn(c, u)); }
};
template <>
struct Arith<double, false> {
    static __device__ __forceinline__ double first(double c, double u) { return __dmul_rn(c, u); }
    static __device__ __forceinline__ double acc(double a, double c, double u) { return __fma_rn(c, u, a); }
};
template <>
struct Arith<float, false> {
    static __device__ __forceinline__ float first(float c, float u) { return __fmul_rn(c, u); }
    static __device__ __forceinline__ float acc(float a, float c, float u) { return __fmaf_rn(c, u, a); }
};

// Star update.  FP64 exact mode adds in coefficient order: centre, then
// (minus, plus) per axis.  The FMA modes add the axis-0 plus neighbour last:
// the tile kernels stream along axis 0, so that operand is the row (plane)
// the previous stage has just produced, and putting it last leaves a single
// dependent FMA between consecutive stages of one step.
template <class T, bool EXACT>
__device__ __forceinline__ T upd1(const Coeffs<T>& c, T C, T m0, T p0) {
    using A = Arith<T, EXACT>;
    T a = A::first(c.c[0], C);
    a = A::acc(a, c.c[1], m0);
    a = A::acc(a, c.c[2], p0);
    return a;
}
template <class T, bool EXACT>
__device__ __forceinline__ T upd2(const Coeffs<T>& c, T C, T m0, T p0, T m1, T p1) {
    using A = Arith<T, EXACT>;
    T a = A::first(c.c[0], C);
    a = A::acc(a, c.c[1], m0);
    if constexpr (EXACT) {
        a = A::acc(a, c.c[2], p0);
        a = A::acc(a, c.c[3], m1);
        a = A::acc(a, c.c[4], p1);
    } else {
        a = A::acc(a, c.c[3], m1);
        a = A::acc(a, c.c[4], p1);
        a = A::acc(a, c.c[2], p0);
    }
    return a;
}
template <class T, bool EXACT>
__device__ __forceinline__ T upd3(const Coeffs<T>& c, T C, T m0, T p0, T m1, T p1, T m2, T p2) {
    using A = Arith<T, EXACT>;
    T a = A::first(c.c[0], C);
    a = A::acc(a, c.c[1], m0);
    if constexpr (EXACT) {
        a = A::acc(a, c.c[2], p0);
        a = A::acc(a, c.c[3], m1);
        a = A::acc(a, c.c[4], p1);
        a = A::acc(a, c.c[5], m2);
        a = A::acc(a, c.c[6], p2);
    } else {
        a = A::acc(a, c.c[3], m1);
        a = A::acc(a, c.c[4], p1);
        a = A::acc(a, c.c[5], m2);
        a = A::acc(a, c.c[6], p2);
        a = A::acc(a, c.c[2], p0);
    }
    return a;
}

// Wrap a storage coordinate of a periodic axis into [0, n).
__device__ __forceinline__ int64_t wrapc(int64_t x, int64_t n) {
    int64_t r = x % n;
    return r < 0 ? r + n : r;
}

// Wrap without 64-bit division for coordinates within one period of [0, n).
__device__ __forceinline__ int64_t wrap_fast(int64_t x, int64_t n) {
    if (x >= 0 && x < n) return x;
    if (x < 0 && x >= -n) return x + n;
    if (x >= n && x < 2 * n) return x - n;
    return wrapc(x, n);
}

// Interior test of one storage coordinate.
__device__ __forceinline__ bool interior_c(int64_t x, int64_t n, bool periodic) {
    return periodic ? true : (x >= 1 && x <= n);
}

// Global loads: plain (through L1) or L2-only (.cg).  The persistent executor
// reads data that other CTAs wrote during the same launch, which must not be
// served from a stale L1 line, so it uses the .cg form.
template <bool CG, class V>
__device__ __forceinline__ V gload(const V* p) {
    if constexpr (CG) return __ldcg(p);
    else return __ldg(p);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_gpu(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Relaxed GPU-scope add: after one fence.acq_rel.gpu (__threadfence) a run of
// these forms a release pattern for every counter, at the cost of one fence
// instead of one per counter.
__device__ __forceinline__ void red_relaxed_add_gpu(int* p, int v) {
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Device status block written by kernels and read by pcot_check.
struct DevStatus {
    int code;      // 0 ok, otherwise a pcot_status value
    int abort;     // set when any CTA gave up; others leave their waits early
    int info[6];   // where it happened (tile id, queue position, ...)
};

constexpr int kStatusTimeout = 6;  // == PCOT_ERR_TIMEOUT
constexpr int kStatusBounds = 7;   // == PCOT_ERR_BOUNDS

// Bounded wait of one thread until *counter reaches 0 (acquire).  Gives up
// after timeout_ns of %globaltimer time, or as soon as another CTA has set
// the abort flag; on giving up it records the status and returns false.
__device__ __forceinline__ bool wait_zero(const int* counter, DevStatus* st, uint64_t timeout_ns,
                                          int info0, int info1) {
    if (ld_acquire_gpu(counter) <= 0) return true;
    const uint64_t t0 = globaltimer_ns();
    unsigned ns = 32;
    for (;;) {
        if (ld_acquire_gpu(counter) <= 0) return true;
        if (*((volatile int*)&st->abort)) return false;
        if (globaltimer_ns() - t0 > timeout_ns) {
            if (atomicCAS(&st->code, 0, kStatusTimeout) == 0) {
                st->info[0] = info0;
                st->info[1] = info1;
            }
            atomicExch(&st->abort, 1);
            return false;
        }
        __nanosleep(ns);
        if (ns < 1024) ns *= 2;
    }
}

}  // namespace pcot
