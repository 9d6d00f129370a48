// Shared device helpers: the complex-double type, fused arithmetic, kernel
// entries of A (paper Eqs. 3, 15, 18) and host error plumbing.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/rss.h"

// ----------------------------------------------------------------- scalars
struct zd {
  double x, y;
};

__host__ __device__ inline zd mkz(double a, double b) { return zd{a, b}; }
__host__ __device__ inline zd operator+(zd a, zd b) { return zd{a.x + b.x, a.y + b.y}; }
__host__ __device__ inline zd operator-(zd a, zd b) { return zd{a.x - b.x, a.y - b.y}; }
__host__ __device__ inline zd operator-(zd a) { return zd{-a.x, -a.y}; }
__host__ __device__ inline zd operator*(zd a, zd b) {
  return zd{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__host__ __device__ inline zd operator*(double s, zd a) { return zd{s * a.x, s * a.y}; }

__host__ __device__ inline double cj(double a) { return a; }
__host__ __device__ inline zd cj(zd a) { return zd{a.x, -a.y}; }
__host__ __device__ inline double abs2(double a) { return a * a; }
__host__ __device__ inline double abs2(zd a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ inline double re(double a) { return a; }
__host__ __device__ inline double re(zd a) { return a.x; }

template <typename T> __host__ __device__ inline T zero();
template <> __host__ __device__ inline double zero<double>() { return 0.0; }
template <> __host__ __device__ inline zd zero<zd>() { return zd{0.0, 0.0}; }
template <typename T> __host__ __device__ inline T from_re(double a);
template <> __host__ __device__ inline double from_re<double>(double a) { return a; }
template <> __host__ __device__ inline zd from_re<zd>(double a) { return zd{a, 0.0}; }

// acc + a * b
__device__ inline double mad(double acc, double a, double b) { return fma(a, b, acc); }
__device__ inline zd mad(zd acc, zd a, zd b) {
  return zd{fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y))};
}
// acc - a * b
__device__ inline double msb(double acc, double a, double b) { return fma(-a, b, acc); }
__device__ inline zd msb(zd acc, zd a, zd b) {
  return zd{fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y))};
}
// acc + conj(a) * b
__device__ inline double madc(double acc, double a, double b) { return fma(a, b, acc); }
__device__ inline zd madc(zd acc, zd a, zd b) {
  return zd{fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y))};
}
// acc - conj(a) * b
__device__ inline double msbc(double acc, double a, double b) { return fma(-a, b, acc); }
__device__ inline zd msbc(zd acc, zd a, zd b) {
  return zd{fma(-a.x, b.x, fma(-a.y, b.y, acc.x)), fma(-a.x, b.y, fma(a.y, b.x, acc.y))};
}
__device__ inline double dv(double a, double b) { return a / b; }
__device__ inline zd dv(zd a, zd b) {
  double d = b.x * b.x + b.y * b.y;
  return zd{(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
__device__ inline double scl(double s, double a) { return s * a; }
__device__ inline zd scl(double s, zd a) { return zd{s * a.x, s * a.y}; }

__device__ inline double shfl_down(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ inline zd shfl_down(zd v, int d) {
  return zd{__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d)};
}
__device__ inline double shfl_xor(double v, int d) { return __shfl_xor_sync(0xffffffffu, v, d); }
__device__ inline zd shfl_xor(zd v, int d) {
  return zd{__shfl_xor_sync(0xffffffffu, v.x, d), __shfl_xor_sync(0xffffffffu, v.y, d)};
}
// loads that bypass L1 (data written by another CTA of the cluster)
__device__ inline double ld_l2(const double* p) { return __ldcg(p); }
__device__ inline zd ld_l2(const zd* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return zd{v.x, v.y};
}

// Asynchronous global -> shared copies (cp.async): a thread issues all its
// copies before waiting once, so a staging loop costs one memory latency
// instead of one per element.  Both addresses must be aligned to the size.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <typename T> __device__ __forceinline__ void cp_async_el(T* smem, const T* gmem) {
  if constexpr (sizeof(T) == 8) cp_async8(smem, gmem);
  else cp_async16(smem, gmem);
}
// wait for this thread's copies; a __syncthreads() must follow before other
// threads read them
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
// close the group of this thread's copies issued since the last commit
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N> __device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ------------------------------------------------------------------ tensor-core fragments
// D += A B on one m16n8k16 tile, bf16 inputs, FP32 accumulators (mma.sync).
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void ldsm_x4(uint32_t* d, const void* smem_row) {
  const unsigned addr = (unsigned)__cvta_generic_to_shared(smem_row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3])
               : "r"(addr));
}

// ------------------------------------------------------------------ tcgen05 (5th-generation tensor cores)
// Operands in shared memory are described by 64-bit matrix descriptors: start
// address, leading-dimension byte offset (LBO: the next 8 entries of K) and
// stride byte offset (SBO: the next 8 rows), both in 16-byte units, version 1,
// no swizzle (K-major core matrices of 8 rows x 16 bytes).  Accumulators live in
// tensor memory (TMEM): row i of a 128-row tile is lane i, each FP32 one column.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: bf16 A and B (K-major), FP32 D, M x N
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// D (+)= A B^T, issued by one thread; accumulate = 0 overwrites D
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// the mbarrier receives one arrival when every tcgen05.mma issued so far by this thread is done
__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// poll phase `parity` of the mbarrier at most `polls` times; false if it never completed
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, long long polls) {
  uint32_t done = 0;
  for (long long it = 0; it < polls && !done; ++it)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
  return done != 0;
}
// warp-wide: allocate / free `cols` TMEM columns (a power of two >= 32); the base address goes to *dst
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(dst)), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(cols) : "memory");
}
// warp-wide: 8 consecutive FP32 columns of this warp's 32 TMEM lanes (lane = thread)
__device__ __forceinline__ void tmem_ld8(uint32_t* v, uint32_t taddr) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// shared-memory writes of this thread (st.shared, completed cp.async) made visible to the tensor core
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// flip the sign of both bf16 values of every register of a fragment
__device__ __forceinline__ void neg_bf16x2(uint32_t* a) {
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] ^= 0x80008000u;
}

// ------------------------------------------------------------------ digit slices, integer only
constexpr int OZ_S = 8;      // digit slices per operand
constexpr int OZ_BITS = 7;   // bits per slice

// A vector x_0..x_{n-1} with max |x| = m 2^e (m in [0.5, 1)) is written as
// x_l = 2^e sum_{p<8} d_{p,l} 2^{-7(p+1)} with signed 7-bit digits (|d_0| <= 128,
// |d_p| <= 64), every digit exact in bf16.  These helpers do it with integer
// operations on the bit patterns (no FP64 instruction).
// |x| as an ordered integer key (non-negative doubles order like their bits)
__device__ __forceinline__ unsigned long long oz_abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
// biased exponent field of the maximum (at least 1), from its key
__device__ __forceinline__ int oz_emax_b(unsigned long long maxkey) {
  const int eb = (int)(maxkey >> 52);
  return eb > 0 ? eb : 1;
}
// x 2^(56 - e) rounded to an integer (ties away from zero), e = emax_b - 1022
__device__ __forceinline__ long long oz_scaled_int(double x, int emax_b) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int eb = (int)((b >> 52) & 0x7FF);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (eb) m |= 1ull << 52;
  const int sh = (eb > 0 ? eb : 1) - emax_b + 3;
  long long X;
  if (sh >= 0) X = (long long)(m << sh);
  else if (sh > -63) X = (long long)((m + (1ull << (-sh - 1))) >> (-sh));
  else X = 0;
  return (b >> 63) ? -X : X;
}
// bf16 bit pattern of a small integer d, |d| <= 128 (exact: conversion instructions)
__device__ __forceinline__ unsigned oz_bf16_int(int d) {
  return (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn((float)d));
}
// the eight digits of X (|X| < 2^56), most significant first, packed for two
// adjacent entries: out[p] = bf16(d_p(X0)) | bf16(d_p(X1)) << 16
__device__ __forceinline__ void oz_digits2(long long X0, long long X1, uint32_t* out) {
  int d0[8], d1[8];
#pragma unroll
  for (int p = 7; p >= 1; --p) {
    d0[p] = (int)(((X0 + 64) & 127) - 64);
    X0 = (X0 - d0[p]) >> 7;
    d1[p] = (int)(((X1 + 64) & 127) - 64);
    X1 = (X1 - d1[p]) >> 7;
  }
  d0[0] = (int)X0;
  d1[0] = (int)X1;
#pragma unroll
  for (int p = 0; p < 8; ++p) out[p] = oz_bf16_int(d0[p]) | (oz_bf16_int(d1[p]) << 16);
}
// An FP32 value holding an integer |g| < 2^22 as an int32, by adding 1.5 2^23 and
// reading the mantissa (one FP32 add and one integer add)
__device__ __forceinline__ int oz_fint(float g) {
  return __float_as_int(g + 12582912.0f) - 0x4B400000;
}

// ------------------------------------------------------------------ E and F on the tensor cores
// One vector x_0..x_{len-1} (x_l = val(l)) shared by G consecutive lanes, cut
// into OZ_S signed 7-bit digit slices as oz_split_row does: 2^e with e the
// exponent of max |x_l|, x_l 2^(56-e) rounded to an integer, digits stored at
// dst[p * ldd + l] for l < lenp (zeros past len).  Every lane of the warp calls
// it (the maximum is a shuffle reduction); inactive groups pass len = 0 and
// store = false.
template <int G, typename VF>
__device__ __forceinline__ void oz_split_vec(VF val, int len, int lenp, uint16_t* dst, int ldd, int* eout,
                                             bool store) {
  // integer operations only (the FP64 pipe is the scarce unit)
  const int gl = threadIdx.x & (G - 1);
  unsigned long long mk = 0;
  for (int l = gl; l < len; l += G) mk = max(mk, oz_abs_bits(val(l)));
#pragma unroll
  for (int d = G / 2; d > 0; d >>= 1)
    mk = max(mk, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mk, d));
  if (!store) return;
  const int eb = oz_emax_b(mk);
  if (gl == 0) *eout = mk ? eb - 1022 : 0;
  for (int l = 2 * gl; l < lenp; l += 2 * G) {
    const long long X0 = l < len ? oz_scaled_int(val(l), eb) : 0;
    const long long X1 = l + 1 < len ? oz_scaled_int(val(l + 1), eb) : 0;
    uint32_t dg[OZ_S];
    oz_digits2(X0, X1, dg);
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) *reinterpret_cast<uint32_t*>(dst + (size_t)p * ldd + l) = dg[p];
  }
}

// W 2^s as a double, W an exact integer (|W| < 2^63): one conversion, the
// power of two added to the exponent field when the result stays normal
__device__ __forceinline__ double oz_ldexp_int(long long W, int s) {
  if (W == 0) return 0.0;
  const double d = (double)W;
  const long long b = __double_as_longlong(d);
  const int eb = (int)((b >> 52) & 0x7FF) + s;
  if (eb > 0 && eb < 2047) return __longlong_as_double(b + ((long long)s << 52));
  return ldexp(d, s);
}

template <typename T> __device__ inline T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = v + shfl_xor(v, d);
  return v;
}

// ----------------------------------------------------------------- kernel entries
struct KParams {
  int kind;
  double h2;        // h^2
  double kappa;
  double diag_re, diag_im;   // A_ii; Lippmann-Schwinger: d in A_ii = 1 + w_i^2 d
  int ncoef;
  double cre[RSS_MAX_COEF], cim[RSS_MAX_COEF];
  double scale, phx, phy;
  const double* w;  // Lippmann-Schwinger: w = kappa sqrt(b) per grid point (iy * side + ix), device
};

// Grid geometry: point (ix, iy) sits at (x0 + ix hg, y0 + iy hg).
struct Geo {
  double x0, y0, hg;
  int side;        // points per grid row
};

__device__ inline zd poly_sum(const KParams& kp, double dx, double dy) {
  // Horner in z = dx + i dy
  zd acc{0.0, 0.0};
  for (int d = kp.ncoef - 1; d >= 0; --d) acc = acc * zd{dx, dy} + zd{kp.cre[d], kp.cim[d]};
  return kp.scale * acc;
}

// K(p1, p2) for p1 != p2 (paper Eq. 3 with Eq. 15 or Eq. 18); p = absolute coordinates.
__device__ inline double kval(const KParams& kp, double x1, double y1, double x2, double y2, double) {
  double dx = x1 - x2, dy = y1 - y2;
  if (kp.kind == RSS_LAPLACE) {
    // -(h^2 / 2 pi) log r = -(h^2 / 4 pi) log r^2
    return (-0.07957747154594767 * kp.h2) * log(fma(dx, dx, dy * dy));
  }
  return poly_sum(kp, dx, dy).x;  // RSS_TEST_RPOLY
}
__device__ inline zd kval(const KParams& kp, double x1, double y1, double x2, double y2, zd) {
  double dx = x1 - x2, dy = y1 - y2;
  if (kp.kind == RSS_HELMHOLTZ || kp.kind == RSS_HELMHOLTZ_LS) {   // (LS: before the weights)
    double kr = kp.kappa * sqrt(fma(dx, dx, dy * dy));
    // h^2 (i/4) (J0 + i Y0) = h^2 (-Y0/4 + i J0/4)
    return zd{-0.25 * kp.h2 * y0(kr), 0.25 * kp.h2 * j0(kr)};
  }
  // RSS_TEST_POLY: conj(w1) w2 p(z1 - z2), w = exp(i (phx x + phy y))
  zd p = poly_sum(kp, dx, dy);
  double s, c;
  sincos(kp.phx * (x2 - x1) + kp.phy * (y2 - y1), &s, &c);
  return p * zd{c, s};
}

// Kernel values by grid displacement.  Every kernel kind here depends only on
// x_i - x_j (the test kernels' phase weights conj(w_i) w_j do too), so on a
// uniform grid K(x_i, x_j) = tab[(iy_i - iy_j + s - 1) (2s - 1) + (ix_i - ix_j + s - 1)].
template <typename T>
__device__ inline T aval_tab(const KParams& kp, const T* __restrict__ tab, int side, int2 a, int2 b) {
  if constexpr (sizeof(T) != sizeof(double)) {
    if (kp.kind == RSS_HELMHOLTZ_LS) {   // A_ij = w_i w_j K_ij, A_ii = 1 + w_i^2 d   (Eqs. 19, 20)
      const double wa = kp.w[a.y * side + a.x];
      if (a.x == b.x && a.y == b.y) return T{1.0 + wa * wa * kp.diag_re, wa * wa * kp.diag_im};
      const double wb = kp.w[b.y * side + b.x];
      return (wa * wb) * tab[(size_t)(a.y - b.y + side - 1) * (2 * side - 1) + (a.x - b.x + side - 1)];
    }
  }
  if (a.x == b.x && a.y == b.y) {
    T d;
    if constexpr (sizeof(T) == sizeof(double)) d = from_re<T>(kp.diag_re);
    else d = T{kp.diag_re, kp.diag_im};
    return d;
  }
  return tab[(size_t)(a.y - b.y + side - 1) * (2 * side - 1) + (a.x - b.x + side - 1)];
}

// ----------------------------------------------------------------- grid barrier
// Barrier over every CTA of a cooperative launch (all CTAs are resident, so each
// one reaches it).  bar[0] counts arrivals, bar[1] is the generation; both start
// at zero, and the count is back at zero after every barrier.  Thread 0 of each
// CTA reads the generation before it arrives; the last CTA to arrive resets the
// count and advances the generation, the others poll it at most `polls` times.
// A wait that runs out sets RSS_ETIMEOUT in *err; every CTA that finds *err set
// (arriving or waiting) leaves the barrier at once, and the barrier returns
// false in every thread of such a CTA (the caller then stops: its results are
// void, and the counters must be zeroed again before the next launch).
__device__ inline bool grid_barrier(unsigned* bar, long long polls, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    volatile int* verr = err;
    int ok = *verr == 0;
    if (ok) {
      const unsigned gen = *vgen;
      __threadfence();   // this CTA's writes are visible before it arrives
      const unsigned arrived = atomicAdd(bar, 1u) + 1u;
      if (arrived == gridDim.x * gridDim.y * gridDim.z) {
        atomicExch(bar, 0u);
        __threadfence();
        atomicAdd(bar + 1, 1u);
      } else {
        long long it = 0;
        while (*vgen == gen && *verr == 0 && it < polls) {
          __nanosleep(64);
          ++it;
        }
        if (*vgen == gen) {
          atomicCAS(err, 0, 5 /* RSS_ETIMEOUT, unless another error came first */);
          ok = 0;
        }
      }
      __threadfence();   // the other CTAs' writes are visible after the barrier
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ----------------------------------------------------------------- host errors
void rss_set_error(const std::string& msg);

#define RSS_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      rss_set_error(std::string("CUDA error: ") + cudaGetErrorString(e_) + " at " + \
                    __FILE__ + ":" + std::to_string(__LINE__));                     \
      return e_ == cudaErrorMemoryAllocation ? RSS_ENOMEM : RSS_ECUDA;              \
    }                                                                               \
  } while (0)

#define RSS_LAUNCHED() RSS_CUDA(cudaGetLastError())

static inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }
