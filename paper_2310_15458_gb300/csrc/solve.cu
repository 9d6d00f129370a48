// Applying the factorization (Section 2.5): x = W_1 .. W_K A_top^{-1} V_K .. V_1 b.
//
// Upward sweep, boxes in factor order (each colour class in one launch):
//   b_R -= T^* b_S;  b_R <- L_R^{-1} P_R b_R;  b_C -= E b_R          (apply V)
// dense top solve, then the downward sweep in reverse order:
//   y_R <- U_R^{-1} (y_R - F y_C);  y_S -= T y_R                       (apply W)
// Boxes of one colour class touch disjoint entries of x, so a class is one
// launch; the right-hand sides are split into chunks of RC columns.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <sstream>
#include <type_traits>

#include "internal.h"
#include "tc_gemm.cuh"

namespace {

constexpr int NT = 256;

template <typename T>
__global__ void k_perm_in(const T* __restrict__ b, int64_t ldb, T* __restrict__ x, int64_t N, int nrhs,
                          const int* __restrict__ u2t) {
  const long long tot = (long long)N * nrhs;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e % N, j = e / N;
    x[u2t[i] + j * N] = b[i + j * ldb];
  }
}

template <typename T>
__global__ void k_perm_out(T* __restrict__ b, int64_t ldb, const T* __restrict__ x, int64_t N, int nrhs,
                           const int* __restrict__ u2t, const int* __restrict__ err) {
  // a grid-barrier wait of the persistent sweeps that ran out (*err != 0) voids
  // the result: every entry becomes NaN rather than a silently wrong number
  const bool bad = err != nullptr && *err != 0;
  const T nan = from_re<T>(__longlong_as_double(0x7FF8000000000000LL));
  const long long tot = (long long)N * nrhs;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e % N, j = e / N;
    b[i + j * ldb] = bad ? nan : x[u2t[i] + j * N];
  }
}

// ------------------------------------------------------------------ sweep kernels
// Rows of C per CTA in the row-chunked kernels; every loop over a factor block
// reads it down columns, so a warp's loads are contiguous.
constexpr int SW_NT = 128;
constexpr int SW_ROWS = 128;
// Per-box kernels whose FP64 work runs one thread per row of R: 64-thread CTAs,
// so the busy warps of consecutive CTAs fall on all four SM sub-partitions
// (an FP64 instruction occupies its sub-partition's pipe for the same time
// with one active lane or 32).
constexpr int SW_NT_R = 64;
constexpr int SW_ROWS_D = 64;   // rows of C per CTA in the downward sweep

// Upward sweep, part 1 (one CTA per box): b_R <- L_R^{-1} P_R (b_R - T^* b_S).
// t = b_R - T^* b_S one thread per row of R; L^{-1} P t as SW_SUB_U sequential
// sums over consecutive parts of R per row (one thread per (row, part): short
// dependency chains, full warps), the parts added in order.  T and L^{-1} P are
// staged in shared memory with coalesced loads when they fit in sm_cap scalars.
constexpr int SW_NT_U = 256;
constexpr int SW_SUB_U = 4;
template <typename T, int RC>
__global__ void __launch_bounds__(SW_NT_U) k_up_r(const BoxRec<T>* __restrict__ recs, T* __restrict__ x, int64_t N,
                                                int nrhs, int sm_cap) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BoxRec<T> R = recs[blockIdx.x];
  const int k = R.k, r = R.r, ldt = k | 1;
  const int q0 = blockIdx.z * RC, nq = min(RC, nrhs - q0);
  T* bS = reinterpret_cast<T*>(smraw);   // k x RC
  T* t = bS + (size_t)k * RC;            // r x RC
  T* ps = t + (size_t)r * RC;            // SW_SUB_U x r x RC: the parts' sums
  T* Ts = ps + (size_t)SW_SUB_U * r * RC;   // T, ld k|1
  T* Ls = Ts + (size_t)ldt * r;          // L^{-1} P, ld r
  const bool stage =
      (size_t)(k + r + SW_SUB_U * r) * RC + (size_t)ldt * r + (size_t)r * r <= (size_t)sm_cap;
  const int tid = threadIdx.x, bs = blockDim.x;
  T* xq = x + (int64_t)q0 * N;
  for (int e = tid; e < k * RC; e += bs) {
    const int s = e / RC, q = e % RC;
    bS[e] = q < nq ? xq[R.idxC[s] + (int64_t)q * N] : zero<T>();
  }
  for (int e = tid; e < r * RC; e += bs) {
    const int j = e / RC, q = e % RC;
    t[e] = q < nq ? xq[R.idxR[j] + (int64_t)q * N] : zero<T>();
  }
  if (stage) {
    for (int e = tid; e < k * r; e += bs) cp_async_el(Ts + (e / k) * ldt + e % k, R.Tm + e);
    for (int e = tid; e < r * r; e += bs) cp_async_el(Ls + e, R.LiP + e);
    cp_async_wait_all();
  }
  __syncthreads();
  const T* Tsrc = stage ? Ts : R.Tm;
  const int tl = stage ? ldt : k;
  const T* Lsrc = stage ? Ls : R.LiP;
  for (int j = tid; j < r; j += bs) {    // t_j -= sum_s conj(T_sj) b_s
    T acc[RC];
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = t[j * RC + q];
    for (int s2 = 0; s2 < k; ++s2) {
      const T tv = Tsrc[s2 + (size_t)j * tl];
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = msbc(acc[q], tv, bS[s2 * RC + q]);
    }
#pragma unroll
    for (int q = 0; q < RC; ++q) t[j * RC + q] = acc[q];
  }
  __syncthreads();
  const int L4 = (r + SW_SUB_U - 1) / SW_SUB_U;
  for (int e = tid; e < SW_SUB_U * r; e += bs) {   // part sc of row j of L^{-1} P t
    const int j = e % r, sc = e / r, l0 = sc * L4, l1 = min(r, l0 + L4);
    T acc[RC];
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = zero<T>();
#pragma unroll 4
    for (int l = l0; l < l1; ++l) {
      const T lv = Lsrc[j + (size_t)l * r];
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = mad(acc[q], lv, t[l * RC + q]);
    }
#pragma unroll
    for (int q = 0; q < RC; ++q) ps[((size_t)sc * r + j) * RC + q] = acc[q];
  }
  __syncthreads();
  for (int e = tid; e < r * RC; e += bs) {   // b_R = the parts added in order
    const int j = e / RC, q = e % RC;
    T p = ps[e];
#pragma unroll
    for (int sc = 1; sc < SW_SUB_U; ++sc) p = p + ps[(size_t)sc * r * RC + e];
    if (q < nq) xq[R.idxR[j] + (int64_t)q * N] = p;
  }
}

// Upward sweep, part 2 (one CTA per SW_ROWS rows of C): b_C -= E b_R.
template <typename T, int RC>
__global__ void __launch_bounds__(SW_NT) k_up_c(const BoxRec<T>* __restrict__ recs, T* __restrict__ x, int64_t N,
                                                int nrhs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BoxRec<T> R = recs[blockIdx.y];
  const int r = R.r, c = R.c, i0 = blockIdx.x * SW_ROWS;
  if (i0 >= c) return;
  const int q0 = blockIdx.z * RC, nq = min(RC, nrhs - q0);
  T* bR = reinterpret_cast<T*>(smraw);   // r x RC
  const int tid = threadIdx.x, bs = blockDim.x;
  T* xq = x + (int64_t)q0 * N;
  for (int e = tid; e < r * RC; e += bs) {
    const int j = e / RC, q = e % RC;
    bR[e] = q < nq ? xq[R.idxR[j] + (int64_t)q * N] : zero<T>();
  }
  __syncthreads();
  const int i1 = min(c, i0 + SW_ROWS);
  for (int i = i0 + tid; i < i1; i += bs) {
    T acc[RC];
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = zero<T>();
    const T* __restrict__ Ei = R.E + i;
#pragma unroll 8
    for (int j = 0; j < r; ++j) {
      const T ev = Ei[(size_t)j * c];
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = mad(acc[q], ev, bR[j * RC + q]);
    }
    const int gi = R.idxC[i];
#pragma unroll
    for (int q = 0; q < RC; ++q)
      if (q < nq) xq[gi + (int64_t)q * N] = xq[gi + (int64_t)q * N] - acc[q];
  }
}

// The end of a box's downward step, given z = y_R - F y_C (shared, r x RC):
// y_R = U^{-1} z into yR (shared) and x, then y_S -= T y_R.  Each product is
// SW_SUB_T sums over consecutive parts of its inner index (rows of U^{-1} from
// the diagonal on, columns of T), one thread per (row, part), added in order.
// ps: SW_SUB_T x max(r, k) x RC scalars of shared memory.  Every thread calls it.
constexpr int SW_SUB_T = 4;
template <typename T, int RC>
__device__ void box_tail(const BoxRec<T>& R, T* xq, int64_t N, int nq, const T* z, T* yR, T* ps,
                         const T* Usrc, const T* Tsrc, int tl, bool l2_reads) {
  const int k = R.k, r = R.r, tid = threadIdx.x, bs = blockDim.x;
  const int L4 = (r + SW_SUB_T - 1) / SW_SUB_T;
  for (int e = tid; e < SW_SUB_T * r; e += bs) {   // part sc of row j of U^{-1} z
    const int j = e % r, sc = e / r, l0 = max(j, sc * L4), l1 = min(r, (sc + 1) * L4);
    T acc[RC];
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = zero<T>();
#pragma unroll 4
    for (int l = l0; l < l1; ++l) {
      const T uv = Usrc[j + (size_t)l * r];
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = mad(acc[q], uv, z[l * RC + q]);
    }
#pragma unroll
    for (int q = 0; q < RC; ++q) ps[((size_t)sc * r + j) * RC + q] = acc[q];
  }
  __syncthreads();
  for (int e = tid; e < r * RC; e += bs) {
    const int j = e / RC, q = e % RC;
    T v = ps[e];
#pragma unroll
    for (int sc = 1; sc < SW_SUB_T; ++sc) v = v + ps[(size_t)sc * r * RC + e];
    yR[e] = v;
    if (q < nq) xq[R.idxR[j] + (int64_t)q * N] = v;
  }
  __syncthreads();
  for (int e = tid; e < SW_SUB_T * k; e += bs) {   // part sc of row s of T y_R
    const int s2 = e % k, sc = e / k, j0 = sc * L4, j1 = min(r, j0 + L4);
    T acc[RC];
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = zero<T>();
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
      const T tv = Tsrc[s2 + (size_t)j * tl];
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = mad(acc[q], tv, yR[j * RC + q]);
    }
#pragma unroll
    for (int q = 0; q < RC; ++q) ps[((size_t)sc * k + s2) * RC + q] = acc[q];
  }
  __syncthreads();
  for (int e = tid; e < k * RC; e += bs) {
    const int s2 = e / RC, q = e % RC;
    T v = ps[e];
#pragma unroll
    for (int sc = 1; sc < SW_SUB_T; ++sc) v = v + ps[(size_t)sc * k * RC + e];
    if (q < nq) {
      const int64_t gs = R.idxC[s2] + (int64_t)q * N;
      xq[gs] = (l2_reads ? ld_l2(xq + gs) : xq[gs]) - v;
    }
  }
  __syncthreads();
}

// Downward sweep (one CTA per SW_ROWS_D rows of C): partial sums of F y_C over
// the CTA's rows from the CTA's block of F^T staged in shared memory (ld
// SW_ROWS_D + 1) when it fits in sm_cap scalars.  Each partial is the sum of
// SW_SUB_D sequential sums over consecutive rows of the chunk, one thread per
// (row of R, part): short dependency chains and full warps.  The last CTA of the
// box to finish (a counter, no waiting) adds the partial sums, forms
// y_R <- U^{-1} (y_R - F y_C) and y_S -= T y_R.  Every CTA has read its rows of
// y_C (which include y_S) before it counts itself in, so the last one may
// overwrite y_S.
constexpr int SW_NT_D = 256;
constexpr int SW_SUB_D = 4;   // sequential sums per 64-row chunk (16 rows each), added in order
template <typename T, int RC>
__global__ void __launch_bounds__(SW_NT_D) k_down(const BoxRec<T>* __restrict__ recs, T* __restrict__ x, int64_t N,
                                                int nrhs, T* __restrict__ part, int* __restrict__ cnt, int nch_max,
                                                int rmax, int sm_cap) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int LDF = SW_ROWS_D + 1;
  const BoxRec<T> R = recs[blockIdx.y];
  // at least one CTA per box: with c = 0 it still forms y_R and y_S
  const int k = R.k, r = R.r, c = R.c, nch = max(1, (c + SW_ROWS_D - 1) / SW_ROWS_D);
  if ((int)blockIdx.x >= nch) return;
  const int i0 = blockIdx.x * SW_ROWS_D, rows = min(SW_ROWS_D, c - i0);
  const int q0 = blockIdx.z * RC, nq = min(RC, nrhs - q0);
  const int tid = threadIdx.x, bs = blockDim.x;
  T* yC = reinterpret_cast<T*>(smraw);   // SW_ROWS_D x RC
  T* ps = yC + (size_t)SW_ROWS_D * RC;     // SW_SUB_D x r x RC: the parts' sums
  T* Fs = ps + (size_t)SW_SUB_D * r * RC;  // rows x r, ld LDF
  __shared__ int s_last;
  T* xq = x + (int64_t)q0 * N;
  const size_t box = (size_t)blockIdx.z * gridDim.y + blockIdx.y;
  const bool stage = (size_t)SW_ROWS_D * RC + (size_t)SW_SUB_D * r * RC + (size_t)LDF * r <= (size_t)sm_cap;
  for (int e = tid; e < rows * RC; e += bs) {
    const int i = e / RC, q = e % RC;
    yC[e] = q < nq ? xq[R.idxC[i0 + i] + (int64_t)q * N] : zero<T>();
  }
  if (stage) {
    for (int e = tid; e < rows * r; e += bs) {
      const int i = e % rows, j = e / rows;
      cp_async_el(Fs + i + (size_t)j * LDF, R.Ft + i0 + i + (size_t)j * c);
    }
    cp_async_wait_all();
  }
  __syncthreads();
  T* pp = part + ((box * nch_max + blockIdx.x) * rmax) * RC;
  constexpr int SUB = SW_ROWS_D / SW_SUB_D;
  for (int e = tid; e < SW_SUB_D * r; e += bs) {   // part sc of row j: rows SUB sc .. SUB sc + SUB - 1
    const int j = e % r, sc = e / r, a0 = sc * SUB, a1 = min(rows, a0 + SUB);
    T acc[RC];
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = zero<T>();
    const T* Fj = stage ? Fs + (size_t)j * LDF : R.Ft + i0 + (size_t)j * c;
#pragma unroll 4
    for (int i = a0; i < a1; ++i) {
      const T fv = Fj[i];
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = mad(acc[q], fv, yC[i * RC + q]);
    }
#pragma unroll
    for (int q = 0; q < RC; ++q) ps[((size_t)sc * r + j) * RC + q] = acc[q];
  }
  __syncthreads();
  for (int e = tid; e < r * RC; e += bs) {
    T p = ps[e];
#pragma unroll
    for (int sc = 1; sc < SW_SUB_D; ++sc) p = p + ps[(size_t)sc * r * RC + e];
    pp[e] = p;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(cnt + box, 1) == nch - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  T* z = yC;                    // r x RC (the shared buffers are free now)
  T* yR = z + (size_t)r * RC;   // r x RC
  T* pt = yR + (size_t)r * RC;  // SW_SUB_T x max(r, k) x RC
  T* Ms = pt + (size_t)SW_SUB_T * max(r, k) * RC;   // U^{-1} (r x r) and T (k x r, ld k|1)
  const int ldt = k | 1;
  const bool stage2 = (size_t)(2 * r + SW_SUB_T * max(r, k)) * RC + (size_t)r * r + (size_t)ldt * r <=
                      (size_t)sm_cap;
  T* Us = Ms;
  T* Ts = Ms + (size_t)r * r;
  for (int e = tid; e < r * RC; e += bs) {
    const int j = e / RC, q = e % RC;
    T sum = zero<T>();
    for (int ch = 0; ch < nch; ++ch) sum = sum + ld_l2(part + ((box * nch_max + ch) * rmax + j) * RC + q);
    z[e] = q < nq ? xq[R.idxR[j] + (int64_t)q * N] - sum : zero<T>();
  }
  if (stage2) {
    for (int e = tid; e < r * r; e += bs) cp_async_el(Us + e, R.Ui + e);
    for (int e = tid; e < k * r; e += bs) cp_async_el(Ts + (e / k) * ldt + e % k, R.Tm + e);
    cp_async_wait_all();
  }
  __syncthreads();
  box_tail<T, RC>(R, xq, N, nq, z, yR, pt, stage2 ? Us : R.Ui, stage2 ? Ts : R.Tm, stage2 ? ldt : k, false);
  if (tid == 0) cnt[box] = 0;   // ready for the next colour class
}

// Downward sweep, one CTA per box (classes with many boxes): the same sums as
// k_down in the same order (per 64-row chunk of C, SW_SUB_D part sums per row of
// F added in order, the chunks added in order, then box_tail), with the chunks
// walked by one CTA and their rows of F^T and of y_C staged by cp.async one
// chunk ahead (two buffers), so no partial sums go through global memory.
template <typename T, int RC>
__host__ __device__ constexpr size_t down_box_sm(int r, int k) {
  return (size_t)r * RC + 2 * (size_t)SW_ROWS_D * RC + 2 * (size_t)(SW_ROWS_D + 1) * r + (size_t)SW_SUB_D * r * RC >
                 (size_t)(3 * r + SW_SUB_T * (r > k ? r : k)) * RC
             ? (size_t)r * RC + 2 * (size_t)SW_ROWS_D * RC + 2 * (size_t)(SW_ROWS_D + 1) * r +
                   (size_t)SW_SUB_D * r * RC
             : (size_t)(3 * r + SW_SUB_T * (r > k ? r : k)) * RC;
}
template <typename T, int RC>
__global__ void __launch_bounds__(SW_NT_D) k_down_box(const BoxRec<T>* __restrict__ recs, T* __restrict__ x, int64_t N,
                                                      int nrhs, int sm_cap) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int LDF = SW_ROWS_D + 1, SUB = SW_ROWS_D / SW_SUB_D;
  const BoxRec<T> R = recs[blockIdx.x];
  const int k = R.k, r = R.r, c = R.c, nch = (c + SW_ROWS_D - 1) / SW_ROWS_D;
  const int q0 = blockIdx.z * RC, nq = min(RC, nrhs - q0);
  const int tid = threadIdx.x, bs = blockDim.x;
  T* xq = x + (int64_t)q0 * N;
  T* zs = reinterpret_cast<T*>(smraw);                 // r x RC: the chunks' sums so far
  T* yC[2] = {zs + (size_t)r * RC, zs + (size_t)r * RC + (size_t)SW_ROWS_D * RC};
  T* Fs[2] = {yC[1] + (size_t)SW_ROWS_D * RC, yC[1] + (size_t)SW_ROWS_D * RC + (size_t)LDF * r};
  T* ps = Fs[1] + (size_t)LDF * r;                     // SW_SUB_D x r x RC
  // copies of chunk ch into buffer b (y_C zero past the chunk's rows and columns)
  auto stage = [&](int ch, int b) {
    const int i0 = ch * SW_ROWS_D, rows = min(SW_ROWS_D, c - i0);
    for (int e = tid; e < rows * r; e += bs) {
      const int i = e % rows, j = e / rows;
      cp_async_el(Fs[b] + i + (size_t)j * LDF, R.Ft + i0 + i + (size_t)j * c);
    }
    for (int e = tid; e < SW_ROWS_D * RC; e += bs) {
      const int ii = e / RC, q = e % RC;
      if (ii < rows && q < nq) cp_async_el(yC[b] + e, xq + R.idxC[i0 + ii] + (int64_t)q * N);
      else yC[b][e] = zero<T>();
    }
    cp_async_commit();
  };
  for (int e = tid; e < r * RC; e += bs) zs[e] = zero<T>();
  if (nch > 0) stage(0, 0);
  for (int ch = 0; ch < nch; ++ch) {
    const int b = ch & 1, rows = min(SW_ROWS_D, c - ch * SW_ROWS_D);
    if (ch + 1 < nch) {
      stage(ch + 1, b ^ 1);   // buffer b ^ 1 was last read before the previous chunk's barrier
      cp_async_wait_group<1>();
    } else {
      cp_async_wait_group<0>();
    }
    __syncthreads();
    for (int e = tid; e < SW_SUB_D * r; e += bs) {
      const int j = e % r, sc = e / r, a0 = sc * SUB, a1 = min(rows, a0 + SUB);
      T acc[RC];
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = zero<T>();
      const T* Fj = Fs[b] + (size_t)j * LDF;
#pragma unroll 4
      for (int i = a0; i < a1; ++i) {
        const T fv = Fj[i];
#pragma unroll
        for (int q = 0; q < RC; ++q) acc[q] = mad(acc[q], fv, yC[b][i * RC + q]);
      }
#pragma unroll
      for (int q = 0; q < RC; ++q) ps[((size_t)sc * r + j) * RC + q] = acc[q];
    }
    __syncthreads();
    for (int e = tid; e < r * RC; e += bs) {   // the chunk's partial, then added to the sum so far
      T p = ps[e];
#pragma unroll
      for (int sc = 1; sc < SW_SUB_D; ++sc) p = p + ps[(size_t)sc * r * RC + e];
      zs[e] = zs[e] + p;
    }
  }
  __syncthreads();   // the chunk buffers are free
  T* z = zs + (size_t)r * RC;
  T* yR = z + (size_t)r * RC;
  T* pt = yR + (size_t)r * RC;
  T* Ms = pt + (size_t)SW_SUB_T * max(r, k) * RC;
  const int ldt = k | 1;
  const bool stage2 = (size_t)(3 * r + SW_SUB_T * max(r, k)) * RC + (size_t)r * r + (size_t)ldt * r <= (size_t)sm_cap;
  T* Us = Ms;
  T* Ts = Ms + (size_t)r * r;
  for (int e = tid; e < r * RC; e += bs) {
    const int j = e / RC, q = e % RC;
    z[e] = q < nq ? xq[R.idxR[j] + (int64_t)q * N] - zs[e] : zero<T>();
  }
  if (stage2) {
    for (int e = tid; e < r * r; e += bs) cp_async_el(Us + e, R.Ui + e);
    for (int e = tid; e < k * r; e += bs) cp_async_el(Ts + (e / k) * ldt + e % k, R.Tm + e);
    cp_async_wait_all();
  }
  __syncthreads();
  box_tail<T, RC>(R, xq, N, nq, z, yR, pt, stage2 ? Us : R.Ui, stage2 ? Ts : R.Tm, stage2 ? ldt : k, false);
}

// ------------------------------------------------------------------ one persistent launch per sweep
// The FP64 sweeps of up to 31 right-hand sides (RC-column chunks, RC = 1, 4, 8)
// as two cooperative launches, one per sweep, instead of two or three launches
// per colour class.  The CTAs walk the colour classes in factor order (upward)
// or reverse order (downward) and meet at a grid barrier between classes.  A
// class with enough boxes for every CTA is taken one box per CTA; a smaller
// class is split by rows of C across CTAs, with one more barrier: upward, the
// boxes' b_R first, then row groups of b_C -= E b_R; downward, partial sums of
// F y_C per group of rows, then per box the rest.  Every sum runs in the same
// order in both forms, for every RC and as in the per-class kernels k_up_r,
// k_up_c and k_down (per row of E: over R ascending; per row of F: a sequential
// sum over each 64-row chunk of C, the chunks added in order), so a column's
// result depends neither on the launch form nor on the other columns.
constexpr int SWP_NT = 128;

// One colour class as the persistent sweeps see it (device array in factor order).
template <typename T> struct SwpClass {
  const BoxRec<T>* recs;
  int nrec, max_k, max_r, max_c;
};
constexpr int SWP_CH = 64;   // rows of C per partial sum of F y_C (fixes the order of the sums, = SW_ROWS_D)

// b_R <- L^{-1} P (b_R - T^* b_S) for one box and RC columns, into bR (shared,
// r x RC) and, when write_x, into x.  Shared memory from sm (sm_cap scalars).
template <typename T, int RC>
__device__ void swp_up_r(const BoxRec<T>& R, T* xq, int64_t N, int nq, T* sm, int sm_cap, T*& bR, bool write_x) {
  const int k = R.k, r = R.r, ldt = k | 1, tid = threadIdx.x, bs = blockDim.x;
  T* bS = sm;
  T* t = bS + (size_t)k * RC;
  bR = t + (size_t)r * RC;
  T* ps = bR + (size_t)r * RC;   // SW_SUB_U x r x RC
  T* Ts = ps + (size_t)SW_SUB_U * r * RC;
  T* Ls = Ts + (size_t)ldt * r;
  const bool stage =
      (size_t)(k + 2 * r + SW_SUB_U * r) * RC + (size_t)ldt * r + (size_t)r * r <= (size_t)sm_cap;
  for (int e = tid; e < k * RC; e += bs) {
    const int s2 = e / RC, q = e % RC;
    bS[e] = q < nq ? ld_l2(xq + R.idxC[s2] + (int64_t)q * N) : zero<T>();
  }
  for (int e = tid; e < r * RC; e += bs) {
    const int j = e / RC, q = e % RC;
    t[e] = q < nq ? ld_l2(xq + R.idxR[j] + (int64_t)q * N) : zero<T>();
  }
  if (stage) {
    for (int e = tid; e < k * r; e += bs) cp_async_el(Ts + (e / k) * ldt + e % k, R.Tm + e);
    for (int e = tid; e < r * r; e += bs) cp_async_el(Ls + e, R.LiP + e);
    cp_async_wait_all();
  }
  __syncthreads();
  const T* Tsrc = stage ? Ts : R.Tm;
  const int tl = stage ? ldt : k;
  const T* Lsrc = stage ? Ls : R.LiP;
  for (int j = tid; j < r; j += bs) {   // t_j -= sum_s conj(T_sj) b_s
    T acc[RC];
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = t[j * RC + q];
    for (int s2 = 0; s2 < k; ++s2) {
      const T tv = Tsrc[s2 + (size_t)j * tl];
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = msbc(acc[q], tv, bS[s2 * RC + q]);
    }
#pragma unroll
    for (int q = 0; q < RC; ++q) t[j * RC + q] = acc[q];
  }
  __syncthreads();
  const int L4 = (r + SW_SUB_U - 1) / SW_SUB_U;
  for (int e = tid; e < SW_SUB_U * r; e += bs) {   // part sc of row j of L^{-1} P t, as k_up_r
    const int j = e % r, sc = e / r, l0 = sc * L4, l1 = min(r, l0 + L4);
    T acc[RC];
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = zero<T>();
#pragma unroll 4
    for (int l = l0; l < l1; ++l) {
      const T lv = Lsrc[j + (size_t)l * r];
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = mad(acc[q], lv, t[l * RC + q]);
    }
#pragma unroll
    for (int q = 0; q < RC; ++q) ps[((size_t)sc * r + j) * RC + q] = acc[q];
  }
  __syncthreads();
  for (int e = tid; e < r * RC; e += bs) {
    const int j = e / RC, q = e % RC;
    T p = ps[e];
#pragma unroll
    for (int sc = 1; sc < SW_SUB_U; ++sc) p = p + ps[(size_t)sc * r * RC + e];
    bR[e] = p;
    if (write_x && q < nq) xq[R.idxR[j] + (int64_t)q * N] = p;
  }
  __syncthreads();
}

// b_C -= E b_R over rows i0 .. i1-1 of C (bR in shared memory).
template <typename T, int RC>
__device__ void swp_up_c(const BoxRec<T>& R, T* xq, int64_t N, int nq, const T* bR, int i0, int i1) {
  const int r = R.r, c = R.c;
  for (int i = i0 + (int)threadIdx.x; i < i1; i += blockDim.x) {
    T acc[RC];
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = zero<T>();
    const T* __restrict__ Ei = R.E + i;
#pragma unroll 8
    for (int j = 0; j < r; ++j) {
      const T ev = Ei[(size_t)j * c];
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = mad(acc[q], ev, bR[j * RC + q]);
    }
    const int gi = R.idxC[i];
#pragma unroll
    for (int q = 0; q < RC; ++q)
      if (q < nq) xq[gi + (int64_t)q * N] = ld_l2(xq + gi + (int64_t)q * N) - acc[q];
  }
}

// Partial sums p(j, ch) = sum over rows of chunk ch of F_ji y_i, for chunks
// ch0 .. ch1-1 of one box, handed to out(j, ch, p[RC]) by the thread that owns
// row j (the same thread for every chunk); each is formed as k_down forms it,
// SW_SUB_D sequential sums over consecutive 16-row parts added in order, so both
// give the same bits.  The chunk's rows of F^T are staged with coalesced copies
// (ld SWP_CH + 1: conflict-free reads down a column).  Uses swp_dn_part_sm(r)
// scalars of sm.
__host__ __device__ constexpr size_t swp_dn_part_sm(int r, int rc) {
  return (size_t)SWP_CH * rc + (size_t)(SWP_CH + 1) * r + (size_t)SW_SUB_D * r * rc;
}
template <typename T, int RC, typename OUT>
__device__ void swp_dn_part(const BoxRec<T>& R, const T* xq, int64_t N, int nq, int ch0, int ch1, T* sm, OUT out) {
  const int r = R.r, c = R.c, tid = threadIdx.x, bs = blockDim.x;
  constexpr int LDF = SWP_CH + 1, SUB = SWP_CH / SW_SUB_D;
  T* yC = sm;                          // SWP_CH x RC
  T* Fs = yC + (size_t)SWP_CH * RC;    // SWP_CH x r, ld LDF
  T* ps = Fs + (size_t)LDF * r;        // SW_SUB_D x r x RC
  for (int ch = ch0; ch < ch1; ++ch) {
    const int i0 = ch * SWP_CH, rows = min(SWP_CH, c - i0);
    __syncthreads();   // the previous chunk's buffers are consumed
    for (int e = tid; e < rows * r; e += bs) {
      const int i = e % rows, j = e / rows;
      cp_async_el(Fs + i + (size_t)j * LDF, R.Ft + i0 + i + (size_t)j * c);
    }
    for (int e = tid; e < SWP_CH * RC; e += bs) {
      const int ii = e / RC, q = e % RC;
      yC[e] = (ii < rows && q < nq) ? ld_l2(xq + R.idxC[i0 + ii] + (int64_t)q * N) : zero<T>();
    }
    cp_async_wait_all();
    __syncthreads();
    for (int e = tid; e < SW_SUB_D * r; e += bs) {
      const int j = e % r, sc = e / r, a0 = sc * SUB, a1 = min(rows, a0 + SUB);
      const T* __restrict__ Fj = Fs + (size_t)j * LDF;
      T acc[RC];
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = zero<T>();
#pragma unroll 4
      for (int ii = a0; ii < a1; ++ii) {
        const T fv = Fj[ii];
#pragma unroll
        for (int q = 0; q < RC; ++q) acc[q] = mad(acc[q], fv, yC[ii * RC + q]);
      }
#pragma unroll
      for (int q = 0; q < RC; ++q) ps[((size_t)sc * r + j) * RC + q] = acc[q];
    }
    __syncthreads();
    for (int j = tid; j < r; j += bs) {
      T p[RC];
#pragma unroll
      for (int q = 0; q < RC; ++q) {
        p[q] = ps[(size_t)j * RC + q];
#pragma unroll
        for (int sc = 1; sc < SW_SUB_D; ++sc) p[q] = p[q] + ps[((size_t)sc * r + j) * RC + q];
      }
      out(j, ch, p);
    }
  }
}

// Given z = y_R - F y_C (zr, shared, r x RC): y_R = U^{-1} z into x, then
// y_S -= T y_R, by box_tail (the order k_down uses).  Uses yR (r x RC) and
// mat_cap scalars at mats: the parts' sums first, then the staged matrices.
template <typename T, int RC>
__device__ void swp_dn_fin(const BoxRec<T>& R, T* xq, int64_t N, int nq, const T* zr, T* yR, T* mats, int mat_cap) {
  const int k = R.k, r = R.r, ldt = k | 1, tid = threadIdx.x, bs = blockDim.x;
  T* pt = mats;
  T* Us = pt + (size_t)SW_SUB_T * max(r, k) * RC;
  T* Ts = Us + (size_t)r * r;
  const bool stage =
      (size_t)SW_SUB_T * max(r, k) * RC + (size_t)r * r + (size_t)ldt * r <= (size_t)max(mat_cap, 0);
  if (stage) {
    for (int e = tid; e < r * r; e += bs) cp_async_el(Us + e, R.Ui + e);
    for (int e = tid; e < k * r; e += bs) cp_async_el(Ts + (e / k) * ldt + e % k, R.Tm + e);
    cp_async_wait_all();
  }
  __syncthreads();
  box_tail<T, RC>(R, xq, N, nq, zr, yR, pt, stage ? Us : R.Ui, stage ? Ts : R.Tm, stage ? ldt : k, true);
}

template <typename T> struct SwpArgs {
  const SwpClass<T>* cls;   // colour classes in factor order
  int ncls;
  T* x;
  int64_t N;
  int nrhs;
  T* part;                  // split classes: partial sums, (z, box, chunk, j, q)
  unsigned* bar;            // grid barrier counters (zeroed before the launch)
  int* err;                 // RSS_ETIMEOUT when a barrier wait runs out
  long long polls;
  int sm_cap;               // scalars of dynamic shared memory
  int spread;               // target work items per CTA and class (the schedule's tuning knob)
};

// Work items of a class: boxes x column chunks (nbz), each box split into ngrp
// groups of cpg whole 64-row chunks of C when that brings the items nearer to
// spread per CTA (ngrp >= 2: the split form), else whole boxes (ngrp = 1).
__device__ __forceinline__ void swp_groups(int max_c, int nbz, int spread, int& nchk, int& ngrp, int& cpg) {
  nchk = (max_c + SWP_CH - 1) / SWP_CH;
  ngrp = min(nchk, (int)(((long long)gridDim.x * spread) / max(nbz, 1)));
  ngrp = max(ngrp, 1);
  cpg = (nchk + ngrp - 1) / ngrp;
  ngrp = (nchk + cpg - 1) / cpg;
}

template <typename T, int RC, bool UP>
__global__ void __launch_bounds__(SWP_NT) k_sweep(SwpArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int nz = (a.nrhs + RC - 1) / RC;
  for (int step = 0; step < a.ncls; ++step) {
    const SwpClass<T> C = a.cls[UP ? step : a.ncls - 1 - step];
    const int nbz = C.nrec * nz;
    int nchk, ngrp, cpg;
    swp_groups(C.max_c, nbz, a.spread, nchk, ngrp, cpg);
    const bool split = ngrp > 1;
    if (UP) {
      if (!split) {
        for (int it = blockIdx.x; it < nbz; it += gridDim.x) {
          const int z = it / C.nrec;
          const BoxRec<T> R = C.recs[it % C.nrec];
          T* xq = a.x + (int64_t)z * RC * a.N;
          const int nq = min(RC, a.nrhs - z * RC);
          T* bR;
          swp_up_r<T, RC>(R, xq, a.N, nq, sm, a.sm_cap, bR, true);
          swp_up_c<T, RC>(R, xq, a.N, nq, bR, 0, R.c);
          __syncthreads();
        }
      } else {
        for (int it = blockIdx.x; it < nbz; it += gridDim.x) {
          const int z = it / C.nrec;
          const BoxRec<T> R = C.recs[it % C.nrec];
          T* bR;
          swp_up_r<T, RC>(R, a.x + (int64_t)z * RC * a.N, a.N, min(RC, a.nrhs - z * RC), sm, a.sm_cap, bR, true);
        }
        if (!grid_barrier(a.bar, a.polls, a.err)) return;
        for (int it = blockIdx.x; it < nbz * ngrp; it += gridDim.x) {
          const int bz = it / ngrp, gi = it % ngrp, z = bz / C.nrec;
          const BoxRec<T> R = C.recs[bz % C.nrec];
          const int i0 = gi * cpg * SWP_CH, i1 = min(R.c, i0 + cpg * SWP_CH);
          if (i0 >= i1) continue;
          T* xq = a.x + (int64_t)z * RC * a.N;
          const int nq = min(RC, a.nrhs - z * RC);
          for (int e = threadIdx.x; e < R.r * RC; e += blockDim.x) {
            const int j = e / RC, q = e % RC;
            sm[e] = q < nq ? ld_l2(xq + R.idxR[j] + (int64_t)q * a.N) : zero<T>();
          }
          __syncthreads();
          swp_up_c<T, RC>(R, xq, a.N, nq, sm, i0, i1);
          __syncthreads();
        }
      }
    } else {
      if (!split) {
        for (int it = blockIdx.x; it < nbz; it += gridDim.x) {
          const int z = it / C.nrec;
          const BoxRec<T> R = C.recs[it % C.nrec];
          T* xq = a.x + (int64_t)z * RC * a.N;
          const int nq = min(RC, a.nrhs - z * RC), r = R.r;
          T* zs = sm;                       // r x RC: running sum of the chunk partials
          T* work = sm + (size_t)r * RC;
          for (int e = threadIdx.x; e < r * RC; e += blockDim.x) zs[e] = zero<T>();
          swp_dn_part<T, RC>(R, xq, a.N, nq, 0, (R.c + SWP_CH - 1) / SWP_CH, work,
                             [&](int j, int, const T* p) {
#pragma unroll
                               for (int q = 0; q < RC; ++q) zs[j * RC + q] = zs[j * RC + q] + p[q];
                             });
          __syncthreads();
          T* zr = work;
          T* yR = zr + (size_t)r * RC;
          for (int e = threadIdx.x; e < r * RC; e += blockDim.x) {
            const int j = e / RC, q = e % RC;
            zr[e] = q < nq ? ld_l2(xq + R.idxR[j] + (int64_t)q * a.N) - zs[e] : zero<T>();
          }
          swp_dn_fin<T, RC>(R, xq, a.N, nq, zr, yR, yR + (size_t)r * RC, a.sm_cap - 3 * r * RC);
        }
      } else {
        const size_t pz = (size_t)C.nrec * nchk * C.max_r * RC;   // part entries per column chunk
        for (int it = blockIdx.x; it < nbz * ngrp; it += gridDim.x) {
          const int bz = it / ngrp, gi = it % ngrp, z = bz / C.nrec, box = bz % C.nrec;
          const BoxRec<T> R = C.recs[box];
          const int nck = (R.c + SWP_CH - 1) / SWP_CH, ch0 = gi * cpg, ch1 = min(nck, ch0 + cpg);
          if (ch0 >= ch1) continue;
          T* pp = a.part + z * pz + (size_t)box * nchk * C.max_r * RC;
          swp_dn_part<T, RC>(R, a.x + (int64_t)z * RC * a.N, a.N, min(RC, a.nrhs - z * RC), ch0, ch1, sm,
                             [&](int j, int ch, const T* p) {
#pragma unroll
                               for (int q = 0; q < RC; ++q) pp[((size_t)ch * C.max_r + j) * RC + q] = p[q];
                             });
          __syncthreads();
        }
        if (!grid_barrier(a.bar, a.polls, a.err)) return;
        for (int it = blockIdx.x; it < nbz; it += gridDim.x) {
          const int z = it / C.nrec, box = it % C.nrec;
          const BoxRec<T> R = C.recs[box];
          T* xq = a.x + (int64_t)z * RC * a.N;
          const int nq = min(RC, a.nrhs - z * RC), r = R.r, nck = (R.c + SWP_CH - 1) / SWP_CH;
          const T* pp = a.part + z * pz + (size_t)box * nchk * C.max_r * RC;
          T* zr = sm;
          T* yR = zr + (size_t)r * RC;
          for (int e = threadIdx.x; e < r * RC; e += blockDim.x) {
            const int j = e / RC, q = e % RC;
            T sum = zero<T>();
            for (int ch = 0; ch < nck; ++ch) sum = sum + ld_l2(pp + ((size_t)ch * C.max_r + j) * RC + q);
            zr[e] = q < nq ? ld_l2(xq + R.idxR[j] + (int64_t)q * a.N) - sum : zero<T>();
          }
          swp_dn_fin<T, RC>(R, xq, a.N, nq, zr, yR, yR + (size_t)r * RC, a.sm_cap - 2 * r * RC);
        }
      }
    }
    if (step + 1 < a.ncls && !grid_barrier(a.bar, a.polls, a.err)) return;
  }
}

// ------------------------------------------------------------------ many right-hand sides on the tensor cores
// Real factors with at least TCN right-hand sides: every product of a sweep is a
// small GEMM (factor block) x (TCN columns of right-hand sides), formed exactly
// from 7-bit digit slices as in the factorization's products: the rows of the
// factor block and the columns of the right-hand sides are scaled by powers of
// two and cut into eight digits (integer operations), the slice products are
// summed exactly by bf16 MMAs with FP32 accumulation, gathered into one int64
// per entry and per K chunk of TCK, and the chunks are added in FP64.  One CTA
// owns one box and TCN columns, so each sweep is one launch per colour class
// with no cross-CTA dependency.
constexpr int TCN = 32, TCM = 64, TCK = 32, TSA = 8 * TCK + 8;   // TSA: bf16 per slice row (16-byte rows)
constexpr int TC_NT = 256;

// C(i, q) receives sum_l A(i, l) B(l, q) for i < M, q < TCN; A(i, l) = aval(i, l),
// B(l, q) = bval(l, q) (FP64).  Every thread of the CTA calls it.
template <typename AF, typename BF, typename OF>
__device__ void tc_gemm32(int M, int K, AF aval, BF bval, OF cout, uint16_t* As, uint16_t* Bs, int* rexp,
                          int* cexp) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, t4 = lane & 3;
  const int m0 = (warp >> 1) * 16, n0 = (warp & 1) * 16;
  const int a_row = lane & 15, a_k = (lane >> 4) * 8;
  const int b_row = ((lane >> 4) << 3) + (lane & 7), b_k = ((lane >> 3) & 1) * 8;
  __syncthreads();   // the caller's shared operands are written (with K = 0 no chunk barrier follows)
  for (int mt = 0; mt < M; mt += TCM) {
    double acc[2][4];
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[ni][e] = 0.0;
    for (int kc = 0; kc < K; kc += TCK) {
      const int kl = min(TCK, K - kc);
      __syncthreads();   // the previous chunk's slices are consumed
      {   // rows of A: 64 rows x 4 lanes
        const int row = tid >> 2, gl = tid & 3, i = mt + row;
        const bool act = i < M;
        unsigned long long mk = 0;
        if (act)
          for (int l = gl; l < kl; l += 4) mk = max(mk, oz_abs_bits(aval(i, kc + l)));
        mk = max(mk, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mk, 1));
        mk = max(mk, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mk, 2));
        const int eb = oz_emax_b(mk);
        if (gl == 0) rexp[row] = eb - 1022;
        uint16_t* dst = As + row * TSA;
        for (int l = 2 * gl; l < TCK; l += 8) {
          const long long X0 = (act && l < kl) ? oz_scaled_int(aval(i, kc + l), eb) : 0;
          const long long X1 = (act && l + 1 < kl) ? oz_scaled_int(aval(i, kc + l + 1), eb) : 0;
          uint32_t dg[8];
          oz_digits2(X0, X1, dg);
#pragma unroll
          for (int p = 0; p < 8; ++p) *reinterpret_cast<uint32_t*>(dst + p * TCK + l) = dg[p];
        }
      }
      {   // columns of B: 32 columns x 8 lanes
        const int col = tid >> 3, gl = tid & 7;
        unsigned long long mk = 0;
        for (int l = gl; l < kl; l += 8) mk = max(mk, oz_abs_bits(bval(kc + l, col)));
#pragma unroll
        for (int d = 1; d < 8; d <<= 1)
          mk = max(mk, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mk, d));
        const int eb = oz_emax_b(mk);
        if (gl == 0) cexp[col] = eb - 1022;
        uint16_t* dst = Bs + col * TSA;
        for (int l = 2 * gl; l < TCK; l += 16) {
          const long long X0 = l < kl ? oz_scaled_int(bval(kc + l, col), eb) : 0;
          const long long X1 = l + 1 < kl ? oz_scaled_int(bval(kc + l + 1, col), eb) : 0;
          uint32_t dg[8];
          oz_digits2(X0, X1, dg);
#pragma unroll
          for (int p = 0; p < 8; ++p) *reinterpret_cast<uint32_t*>(dst + p * TCK + l) = dg[p];
        }
      }
      __syncthreads();
      long long W[2][4];
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int e = 0; e < 4; ++e) W[ni][e] = 0;
#pragma unroll 1
      for (int u = 0; u < 8; u += 2) {   // groups u, u + 1 together (|G| < 2^22)
        float c0[2][4], c1[2][4];
#pragma unroll
        for (int ni = 0; ni < 2; ++ni)
#pragma unroll
          for (int e = 0; e < 4; ++e) c0[ni][e] = c1[ni][e] = 0.f;
        for (int p = 0; p <= u + 1; ++p) {
          const uint16_t* Ab = As + p * TCK + (m0 + a_row) * TSA + a_k;
#pragma unroll
          for (int kk = 0; kk < TCK; kk += 16) {
            uint32_t af[4], bq[4];
            ldsm_x4(af, Ab + kk);
            ldsm_x4(bq, Bs + (u + 1 - p) * TCK + (n0 + b_row) * TSA + b_k + kk);
            mma_bf16(c1[0], af, bq);
            mma_bf16(c1[1], af, bq + 2);
            if (p <= u) {
              ldsm_x4(bq, Bs + (u - p) * TCK + (n0 + b_row) * TSA + b_k + kk);
              mma_bf16(c0[0], af, bq);
              mma_bf16(c0[1], af, bq + 2);
            }
          }
        }
        const int sh = 32 - 7 * u;
#pragma unroll
        for (int ni = 0; ni < 2; ++ni)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const long long gv = (long long)(oz_fint(c0[ni][e]) * 128 + oz_fint(c1[ni][e]));
            W[ni][e] += sh >= 0 ? (gv << sh) : ((gv + (1LL << (-sh - 1))) >> (-sh));
          }
      }
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int row = m0 + gq + (e >= 2 ? 8 : 0), col = n0 + ni * 8 + 2 * t4 + (e & 1);
          acc[ni][e] += oz_ldexp_int(W[ni][e], rexp[row] + cexp[col] - 53);
        }
    }
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = m0 + gq + (e >= 2 ? 8 : 0), col = n0 + ni * 8 + 2 * t4 + (e & 1);
        if (mt + row < M) cout(mt + row, col, acc[ni][e]);
      }
  }
  __syncthreads();
}

__device__ __forceinline__ size_t tc_smem_head() {
  return (size_t)(TCM + TCN) * TSA * sizeof(uint16_t);
}

// Slices of the rows of E (K = r), 64 rows per CTA, four lanes per row.
__global__ void __launch_bounds__(TC_NT) k_slice_e(const BoxRec<double>* __restrict__ recs,
                                                   const SliceRec* __restrict__ sl) {
  const BoxRec<double> R = recs[blockIdx.x];
  const SliceRec S = sl[blockIdx.x];
  const int i = blockIdx.y * 64 + (int)threadIdx.x / 4, c = R.c, r = R.r;
  if (blockIdx.y * 64 >= c) return;
  const bool act = i < c;
  const double* E = R.E;
  oz_split_vec<4>([&](int l) { return E[i + (size_t)l * c]; }, act ? r : 0, S.kp,
                  S.Esl + (size_t)(act ? i : 0) * OZ_S * S.kp, S.kp, S.Eexp + (act ? i : 0), act);
}

// Slices of the rows of F (columns of F^T, K = c), one warp per row.
__global__ void __launch_bounds__(TC_NT) k_slice_f(const BoxRec<double>* __restrict__ recs,
                                                   const SliceRec* __restrict__ sl) {
  const BoxRec<double> R = recs[blockIdx.x];
  const SliceRec S = sl[blockIdx.x];
  const int j = blockIdx.y * (TC_NT / 32) + (int)threadIdx.x / 32, c = R.c, r = R.r;
  if (blockIdx.y * (TC_NT / 32) >= r) return;
  const bool act = j < r;
  const double* Fc = R.Ft + (size_t)(act ? j : 0) * c;
  oz_split_vec<32>([&](int l) { return Fc[l]; }, act ? c : 0, S.cp, S.Fsl + (size_t)(act ? j : 0) * OZ_S * S.cp,
                   S.cp, S.Fexp + (act ? j : 0), act);
}

// C(i, q) receives sum_l A(i, l) B(l, q) for i < M, q < TCN, with the rows of A
// given as precomputed slices (row i at Asl + i * OZ_S * ka, scale 2^Aexp[i],
// zero past K) and B(l, q) = bval(l, q) in FP64, cut here under one scale per
// column over the whole K.  With both scales fixed along K, the eight group
// sums stay exact in FP32 for 384 entries of K and are gathered into one int64
// per entry (|W| <= K 2^53, K < 1024); K is staged in chunks of TCK.  Every
// thread of the CTA calls it.
template <typename BF, typename OF>
__device__ void tc_gemm_sl(int M, int ka, const uint16_t* __restrict__ Asl, const int* __restrict__ Aexp, BF bval,
                           OF cout, uint16_t* As, uint16_t* Bs, int* rexp, int* cexp, int* ceb) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, t4 = lane & 3;
  const int m0 = (warp >> 1) * 16, n0 = (warp & 1) * 16;
  const int a_row = lane & 15, a_k = (lane >> 4) * 8;
  const int b_row = ((lane >> 4) << 3) + (lane & 7), b_k = ((lane >> 3) & 1) * 8;
  {   // column scales of B over the whole K (zero past it)
    const int col = tid >> 3, gl = tid & 7;
    unsigned long long mk = 0;
    for (int l = gl; l < ka; l += 8) mk = max(mk, oz_abs_bits(bval(l, col)));
#pragma unroll
    for (int d = 1; d < 8; d <<= 1)
      mk = max(mk, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mk, d));
    const int eb = oz_emax_b(mk);
    if (gl == 0) {
      ceb[col] = eb;
      cexp[col] = mk ? eb - 1022 : 0;
    }
  }
  for (int mt = 0; mt < M; mt += TCM) {
    float acc[OZ_S][2][4];
    long long W[2][4];
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        W[ni][e] = 0;
#pragma unroll
        for (int u = 0; u < OZ_S; ++u) acc[u][ni][e] = 0.f;
      }
    auto gather = [&]() {
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          long long w = W[ni][e];
#pragma unroll
          for (int u = 0; u < OZ_S; u += 2) {
            const long long gv = (long long)(oz_fint(acc[u][ni][e]) * 128 + oz_fint(acc[u + 1][ni][e]));
            const int sh = 32 - OZ_BITS * u;
            w += sh >= 0 ? (gv << sh) : ((gv + (1LL << (-sh - 1))) >> (-sh));
            acc[u][ni][e] = acc[u + 1][ni][e] = 0.f;
          }
          W[ni][e] = w;
        }
    };
    for (int kc = 0; kc < ka; kc += TCK) {
      const int kl = min(TCK, ka - kc), cpr = OZ_S * (kl / 8);   // ka is a multiple of 16
      __syncthreads();   // the previous chunk is consumed (and the column scales are visible)
      for (int e = tid; e < TCM * cpr; e += TC_NT) {   // rows of A: slices p, entries kc .. kc + kl
        const int row = e / cpr, rem = e % cpr, p = rem / (kl / 8), ch = rem % (kl / 8);
        uint16_t* d = As + row * TSA + p * TCK + ch * 8;
        if (mt + row < M)
          cp_async16(d, Asl + (size_t)(mt + row) * OZ_S * ka + (size_t)p * ka + kc + ch * 8);
        else
          *reinterpret_cast<uint4*>(d) = make_uint4(0, 0, 0, 0);
      }
      {   // columns of B: 32 columns x 8 lanes, two entries per lane and step
        const int col = tid >> 3, gl = tid & 7, eb = ceb[col];
        uint16_t* dst = Bs + col * TSA;
        for (int l = 2 * gl; l < TCK; l += 16) {
          const long long X0 = l < kl ? oz_scaled_int(bval(kc + l, col), eb) : 0;
          const long long X1 = l + 1 < kl ? oz_scaled_int(bval(kc + l + 1, col), eb) : 0;
          uint32_t dg[8];
          oz_digits2(X0, X1, dg);
#pragma unroll
          for (int p = 0; p < 8; ++p) *reinterpret_cast<uint32_t*>(dst + p * TCK + l) = dg[p];
        }
      }
      cp_async_wait_all();
      __syncthreads();
      for (int kk = 0; kk < kl; kk += 16) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {   // slices q = 4h .. 4h + 3 of B, then every A slice p <= 7 - q
          uint32_t bq[4][4];
#pragma unroll
          for (int q = 0; q < 4; ++q) ldsm_x4(bq[q], Bs + (n0 + b_row) * TSA + (4 * h + q) * TCK + kk + b_k);
#pragma unroll
          for (int p = 0; p + 4 * h < OZ_S; ++p) {
            uint32_t af[4];
            ldsm_x4(af, As + (m0 + a_row) * TSA + p * TCK + kk + a_k);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (p + 4 * h + q < OZ_S) {
                mma_bf16(acc[p + 4 * h + q][0], af, bq[q]);
                mma_bf16(acc[p + 4 * h + q][1], af, bq[q] + 2);
              }
          }
        }
      }
      if ((kc / TCK + 1) % 12 == 0 && kc + TCK < ka) gather();   // 12 chunks: 384 entries of K
    }
    gather();
    if (tid < TCM) rexp[tid] = mt + tid < M ? Aexp[mt + tid] : 0;
    __syncthreads();
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = m0 + gq + (e >= 2 ? 8 : 0), col = n0 + ni * 8 + 2 * t4 + (e & 1);
        if (mt + row < M) cout(mt + row, col, oz_ldexp_int(W[ni][e], rexp[row] + cexp[col] - 53));
      }
  }
  __syncthreads();
}

// Upward sweep of one box for TCN right-hand-side columns:
// t = b_R - T^* b_S, b_R = L^{-1} P t, b_C -= E b_R.
__global__ void __launch_bounds__(TC_NT, 2) k_up_tc(const BoxRec<double>* __restrict__ recs,
                                                    const SliceRec* __restrict__ sl, double* __restrict__ x,
                                                    int64_t N, int nrhs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BoxRec<double> R = recs[blockIdx.x];
  const int k = R.k, r = R.r, c = R.c;
  const int q0 = blockIdx.y * TCN, nq = min(TCN, nrhs - q0);
  uint16_t* As = reinterpret_cast<uint16_t*>(smraw);
  uint16_t* Bs = As + TCM * TSA;
  double* bS = reinterpret_cast<double*>(smraw + tc_smem_head());   // k x TCN
  double* t = bS + (size_t)k * TCN;                                  // r x TCN
  double* u = t + (size_t)r * TCN;                                   // r x TCN
  __shared__ int rexp[TCM], cexp[TCN], ceb[TCN];
  const int tid = threadIdx.x, bs = blockDim.x;
  double* xq = x + (int64_t)q0 * N;
  for (int e = tid; e < k * TCN; e += bs) {
    const int s2 = e / TCN, q = e % TCN;
    bS[e] = q < nq ? xq[R.idxC[s2] + (int64_t)q * N] : 0.0;
  }
  for (int e = tid; e < r * TCN; e += bs) {
    const int j = e / TCN, q = e % TCN;
    t[e] = q < nq ? xq[R.idxR[j] + (int64_t)q * N] : 0.0;
  }
  const double* __restrict__ Tm = R.Tm;
  const double* __restrict__ LiP = R.LiP;
  const double* __restrict__ E = R.E;
  tc_gemm32(r, k, [&](int i, int l) { return Tm[l + (size_t)i * k]; }, [&](int l, int q) { return bS[l * TCN + q]; },
            [&](int i, int q, double v) { t[i * TCN + q] -= v; }, As, Bs, rexp, cexp);
  tc_gemm32(r, r, [&](int i, int l) { return LiP[i + (size_t)l * r]; }, [&](int l, int q) { return t[l * TCN + q]; },
            [&](int i, int q, double v) { u[i * TCN + q] = v; }, As, Bs, rexp, cexp);
  for (int e = tid; e < r * TCN; e += bs) {
    const int j = e / TCN, q = e % TCN;
    if (q < nq) xq[R.idxR[j] + (int64_t)q * N] = u[e];
  }
  auto sub_c = [&](int i, int q, double v) {
    if (q < nq) {
      const int64_t gi = R.idxC[i] + (int64_t)q * N;
      xq[gi] = xq[gi] - v;
    }
  };
  if (sl != nullptr) {
    const SliceRec S = sl[blockIdx.x];
    tc_gemm_sl(c, S.kp, S.Esl, S.Eexp, [&](int l, int q) { return l < r ? u[l * TCN + q] : 0.0; }, sub_c, As, Bs,
               rexp, cexp, ceb);
  } else {
    tc_gemm32(c, r, [&](int i, int l) { return E[i + (size_t)l * c]; }, [&](int l, int q) { return u[l * TCN + q]; },
              sub_c, As, Bs, rexp, cexp);
  }
}

// Downward sweep of one box for TCN columns: z = y_R - F y_C, y_R = U^{-1} z,
// y_S -= T y_R.
__global__ void __launch_bounds__(TC_NT, 2) k_down_tc(const BoxRec<double>* __restrict__ recs,
                                                      const SliceRec* __restrict__ sl, double* __restrict__ x,
                                                      int64_t N, int nrhs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BoxRec<double> R = recs[blockIdx.x];
  const int k = R.k, r = R.r, c = R.c;
  const int q0 = blockIdx.y * TCN, nq = min(TCN, nrhs - q0);
  uint16_t* As = reinterpret_cast<uint16_t*>(smraw);
  uint16_t* Bs = As + TCM * TSA;
  double* z = reinterpret_cast<double*>(smraw + tc_smem_head());   // r x TCN
  double* yR = z + (size_t)r * TCN;                                 // r x TCN
  __shared__ int rexp[TCM], cexp[TCN], ceb[TCN];
  const int tid = threadIdx.x, bs = blockDim.x;
  double* xq = x + (int64_t)q0 * N;
  for (int e = tid; e < r * TCN; e += bs) {
    const int j = e / TCN, q = e % TCN;
    z[e] = q < nq ? xq[R.idxR[j] + (int64_t)q * N] : 0.0;
  }
  const double* __restrict__ Ft = R.Ft;
  const double* __restrict__ Ui = R.Ui;
  const double* __restrict__ Tm = R.Tm;
  const int* __restrict__ idxC = R.idxC;
  if (sl != nullptr) {
    const SliceRec S = sl[blockIdx.x];
    tc_gemm_sl(r, S.cp, S.Fsl, S.Fexp,
               [&](int i, int q) { return (i < c && q < nq) ? xq[idxC[i] + (int64_t)q * N] : 0.0; },
               [&](int j, int q, double v) { z[j * TCN + q] -= v; }, As, Bs, rexp, cexp, ceb);
  } else {
    tc_gemm32(r, c, [&](int j, int i) { return Ft[i + (size_t)j * c]; },
              [&](int i, int q) { return q < nq ? xq[idxC[i] + (int64_t)q * N] : 0.0; },
              [&](int j, int q, double v) { z[j * TCN + q] -= v; }, As, Bs, rexp, cexp);
  }
  tc_gemm32(r, r, [&](int j, int l) { return Ui[j + (size_t)l * r]; }, [&](int l, int q) { return z[l * TCN + q]; },
            [&](int j, int q, double v) { yR[j * TCN + q] = v; }, As, Bs, rexp, cexp);
  for (int e = tid; e < r * TCN; e += bs) {
    const int j = e / TCN, q = e % TCN;
    if (q < nq) xq[R.idxR[j] + (int64_t)q * N] = yR[e];
  }
  tc_gemm32(k, r, [&](int s2, int j) { return Tm[s2 + (size_t)j * k]; }, [&](int j, int q) { return yR[j * TCN + q]; },
            [&](int s2, int q, double v) {
              if (q < nq) {
                const int64_t gs = idxC[s2] + (int64_t)q * N;
                xq[gs] = xq[gs] - v;
              }
            },
            As, Bs, rexp, cexp);
}

// Complex factors with at least ZCN right-hand sides: the products of both sweeps
// as complex digit-slice GEMMs on the tensor cores (tc_gemm_c), one CTA per box
// and ZCN columns; the vectors of the box stay in shared memory between them.
__device__ __forceinline__ size_t tcz_head() { return (size_t)(ZCM + ZCN) * ZSA * sizeof(uint16_t); }
inline size_t tcz_smem_up(int k, int r) { return (size_t)(ZCM + ZCN) * ZSA * 2 + sizeof(zd) * (size_t)(k + 2 * r) * ZCN; }
inline size_t tcz_smem_down(int r) { return (size_t)(ZCM + ZCN) * ZSA * 2 + sizeof(zd) * (size_t)(2 * r) * ZCN; }
constexpr size_t TCZ_SMEM_MAX = 220 * 1024;

// t = b_R - T^* b_S, b_R = L^{-1} P t, b_C -= E b_R.
__global__ void __launch_bounds__(TC_NT) k_up_tcz(const BoxRec<zd>* __restrict__ recs, zd* __restrict__ x,
                                                  int64_t N, int nrhs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BoxRec<zd> R = recs[blockIdx.x];
  const int k = R.k, r = R.r, c = R.c;
  const int q0 = blockIdx.y * ZCN, nq = min(ZCN, nrhs - q0);
  uint16_t* As = reinterpret_cast<uint16_t*>(smraw);
  uint16_t* Bs = As + ZCM * ZSA;
  zd* bS = reinterpret_cast<zd*>(smraw + tcz_head());   // k x ZCN
  zd* t = bS + (size_t)k * ZCN;                           // r x ZCN
  zd* u = t + (size_t)r * ZCN;                            // r x ZCN
  __shared__ int rexp[ZCM], cexp[ZCN];
  const int tid = threadIdx.x, bs = blockDim.x;
  zd* xq = x + (int64_t)q0 * N;
  for (int e = tid; e < k * ZCN; e += bs) {
    const int s2 = e / ZCN, q = e % ZCN;
    bS[e] = q < nq ? xq[R.idxC[s2] + (int64_t)q * N] : zero<zd>();
  }
  for (int e = tid; e < r * ZCN; e += bs) {
    const int j = e / ZCN, q = e % ZCN;
    t[e] = q < nq ? xq[R.idxR[j] + (int64_t)q * N] : zero<zd>();
  }
  __syncthreads();   // (tc_gemm_c synchronises per K chunk; K = k may be 0)
  const zd* __restrict__ Tm = R.Tm;
  const zd* __restrict__ LiP = R.LiP;
  const zd* __restrict__ E = R.E;
  tc_gemm_c(r, k, [&](int i, int l) { return cj(Tm[l + (size_t)i * k]); }, [&](int l, int q) { return bS[l * ZCN + q]; },
            [&](int i, int q, zd v) { t[i * ZCN + q] = t[i * ZCN + q] - v; }, As, Bs, rexp, cexp);
  tc_gemm_c(r, r, [&](int i, int l) { return LiP[i + (size_t)l * r]; }, [&](int l, int q) { return t[l * ZCN + q]; },
            [&](int i, int q, zd v) { u[i * ZCN + q] = v; }, As, Bs, rexp, cexp);
  for (int e = tid; e < r * ZCN; e += bs) {
    const int j = e / ZCN, q = e % ZCN;
    if (q < nq) xq[R.idxR[j] + (int64_t)q * N] = u[e];
  }
  tc_gemm_c(c, r, [&](int i, int l) { return E[i + (size_t)l * c]; }, [&](int l, int q) { return u[l * ZCN + q]; },
            [&](int i, int q, zd v) {
              if (q < nq) {
                const int64_t gi = R.idxC[i] + (int64_t)q * N;
                xq[gi] = xq[gi] - v;
              }
            },
            As, Bs, rexp, cexp);
}

// z = y_R - F y_C, y_R = U^{-1} z, y_S -= T y_R.
__global__ void __launch_bounds__(TC_NT) k_down_tcz(const BoxRec<zd>* __restrict__ recs, zd* __restrict__ x,
                                                    int64_t N, int nrhs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BoxRec<zd> R = recs[blockIdx.x];
  const int k = R.k, r = R.r, c = R.c;
  const int q0 = blockIdx.y * ZCN, nq = min(ZCN, nrhs - q0);
  uint16_t* As = reinterpret_cast<uint16_t*>(smraw);
  uint16_t* Bs = As + ZCM * ZSA;
  zd* z = reinterpret_cast<zd*>(smraw + tcz_head());   // r x ZCN
  zd* yR = z + (size_t)r * ZCN;                          // r x ZCN
  __shared__ int rexp[ZCM], cexp[ZCN];
  const int tid = threadIdx.x, bs = blockDim.x;
  zd* xq = x + (int64_t)q0 * N;
  for (int e = tid; e < r * ZCN; e += bs) {
    const int j = e / ZCN, q = e % ZCN;
    z[e] = q < nq ? xq[R.idxR[j] + (int64_t)q * N] : zero<zd>();
  }
  __syncthreads();
  const zd* __restrict__ Ft = R.Ft;
  const zd* __restrict__ Ui = R.Ui;
  const zd* __restrict__ Tm = R.Tm;
  const int* __restrict__ idxC = R.idxC;
  tc_gemm_c(r, c, [&](int j, int i) { return Ft[i + (size_t)j * c]; },
            [&](int i, int q) { return q < nq ? xq[idxC[i] + (int64_t)q * N] : zero<zd>(); },
            [&](int j, int q, zd v) { z[j * ZCN + q] = z[j * ZCN + q] - v; }, As, Bs, rexp, cexp);
  tc_gemm_c(r, r, [&](int j, int l) { return Ui[j + (size_t)l * r]; }, [&](int l, int q) { return z[l * ZCN + q]; },
            [&](int j, int q, zd v) { yR[j * ZCN + q] = v; }, As, Bs, rexp, cexp);
  for (int e = tid; e < r * ZCN; e += bs) {
    const int j = e / ZCN, q = e % ZCN;
    if (q < nq) xq[R.idxR[j] + (int64_t)q * N] = yR[e];
  }
  tc_gemm_c(k, r, [&](int s2, int j) { return Tm[s2 + (size_t)j * k]; }, [&](int j, int q) { return yR[j * ZCN + q]; },
            [&](int s2, int q, zd v) {
              if (q < nq) {
                const int64_t gs = idxC[s2] + (int64_t)q * N;
                xq[gs] = xq[gs] - v;
              }
            },
            As, Bs, rexp, cexp);
}

// Top block: x_top <- A_top^{-1} x_top with the inverse formed at factor time.
template <typename T>
__global__ void k_top_gather(const int* __restrict__ idx, int n, const T* __restrict__ x, int64_t N, int nrhs,
                             T* __restrict__ z) {
  const long long tot = (long long)n * nrhs;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n);
    const long long q = e / n;
    z[e] = x[idx[i] + q * N];
  }
}

template <typename T, int RC>
__global__ void __launch_bounds__(SW_NT) k_top_gemv(const T* __restrict__ Ainv, const int* __restrict__ idx, int n,
                                                    const T* __restrict__ z, T* __restrict__ x, int64_t N, int nrhs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* zs = reinterpret_cast<T*>(smraw);   // n x RC
  const int q0 = blockIdx.y * RC, nq = min(RC, nrhs - q0);
  for (int e = threadIdx.x; e < n * RC; e += blockDim.x) {
    const int j = e / RC, q = e % RC;
    zs[e] = q < nq ? z[j + (int64_t)(q0 + q) * n] : zero<T>();
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T acc[RC];
#pragma unroll
  for (int q = 0; q < RC; ++q) acc[q] = zero<T>();
#pragma unroll 8
  for (int j = 0; j < n; ++j) {
    const T av = Ainv[i + (size_t)j * n];
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = mad(acc[q], av, zs[j * RC + q]);
  }
#pragma unroll
  for (int q = 0; q < RC; ++q)
    if (q < nq) x[idx[i] + (int64_t)(q0 + q) * N] = acc[q];
}

// Dense top solve, blocked by 32: one warp solves each diagonal block (no
// block-wide barrier per row), then all threads update the rows below (above).
template <typename T, int RC>
__global__ void __launch_bounds__(1024) k_top_solve(const T* __restrict__ LU, const int* __restrict__ piv,
                                                    const int* __restrict__ idx, int n, T* __restrict__ x,
                                                    int64_t N, int nrhs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* z = reinterpret_cast<T*>(smraw);   // n x RC
  const int q0 = blockIdx.x * RC, nq = min(RC, nrhs - q0);
  const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, warp = tid >> 5;
  T* xq = x + (int64_t)q0 * N;
  for (int e = tid; e < n * RC; e += bs) {
    const int i = e / RC, q = e % RC;
    z[e] = q < nq ? xq[idx[i] + (int64_t)q * N] : zero<T>();
  }
  __syncthreads();
  if (tid < RC)
    for (int j = 0; j < n; ++j) {
      const int p = piv[j];
      if (p != j) {
        const T t = z[j * RC + tid];
        z[j * RC + tid] = z[p * RC + tid];
        z[p * RC + tid] = t;
      }
    }
  __syncthreads();
  // forward: unit lower L
  for (int jb = 0; jb < n; jb += 32) {
    const int je = min(n, jb + 32);
    if (warp == 0) {
      for (int j = jb; j < je; ++j) {
        const int l = jb + lane;
        if (l > j && l < je)
          for (int q = 0; q < RC; ++q) z[l * RC + q] = msb(z[l * RC + q], LU[l + (size_t)j * n], z[j * RC + q]);
        __syncwarp();
      }
    }
    __syncthreads();
    for (int e = tid; e < (n - je) * RC; e += bs) {
      const int l = je + e / RC, q = e % RC;
      T acc = z[l * RC + q];
      for (int j = jb; j < je; ++j) acc = msb(acc, LU[l + (size_t)j * n], z[j * RC + q]);
      z[l * RC + q] = acc;
    }
    __syncthreads();
  }
  // backward: upper U
  for (int je = n; je > 0; je -= 32) {
    const int jb = max(0, je - 32);
    if (warp == 0) {
      for (int j = je - 1; j >= jb; --j) {
        if (lane == 0)
          for (int q = 0; q < RC; ++q) z[j * RC + q] = dv(z[j * RC + q], LU[j + (size_t)j * n]);
        __syncwarp();
        const int l = jb + lane;
        if (l < j)
          for (int q = 0; q < RC; ++q) z[l * RC + q] = msb(z[l * RC + q], LU[l + (size_t)j * n], z[j * RC + q]);
        __syncwarp();
      }
    }
    __syncthreads();
    for (int e = tid; e < jb * RC; e += bs) {
      const int l = e / RC, q = e % RC;
      T acc = z[l * RC + q];
      for (int j = jb; j < je; ++j) acc = msb(acc, LU[l + (size_t)j * n], z[j * RC + q]);
      z[l * RC + q] = acc;
    }
    __syncthreads();
  }
  for (int e = tid; e < n * RC; e += bs) {
    const int i = e / RC, q = e % RC;
    if (q < nq) xq[idx[i] + (int64_t)q * N] = z[e];
  }
}

__global__ void k_iota(int* v, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = i;
}
template <typename T> __global__ void k_identity(T* A, int n) {
  const long long tot = (long long)n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x)
    A[e] = (e % n == e / n) ? from_re<T>(1.0) : zero<T>();
}

// Workspace of the sweeps for nrhs right-hand sides in chunks of rc columns:
// the downward sweep's partial sums, one counter per box, the gathered top block.
// (The persistent sweeps use the same partial-sum region, with 64-row chunks,
// and four ints at bar_off: grid barrier counters and the timeout flag.)
struct SweepWs {
  size_t cnt_off = 0, bar_off = 0, topz_off = 0, bytes = 0;
};

template <typename T> SweepWs sweep_ws(const rss_factorization* f, int64_t nrhs, int rc) {
  const size_t nz = cdiv(nrhs, rc);
  size_t part = 0, cnt = 0;
  for (const Batch& b : f->batches) {
    part = std::max(part, (size_t)b.nrec * cdiv(b.max_c, SW_ROWS_D) * b.max_r);
    cnt = std::max(cnt, (size_t)b.nrec);
  }
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  SweepWs w;
  w.cnt_off = al(sizeof(T) * part * nz * rc);
  w.bar_off = w.cnt_off + al(sizeof(int) * cnt * nz);
  w.topz_off = w.bar_off + al(sizeof(int) * 4);
  w.bytes = w.topz_off + al(sizeof(T) * (size_t)f->ntop * nz * rc);
  return w;
}

int rhs_chunk(int64_t nrhs) { return nrhs == 1 ? 1 : nrhs <= 4 ? 4 : 8; }

// Top block: x_top <- A_top^{-1} x_top (gathered, one product, scattered back).
template <typename T, int RC>
rss_status top_apply(const rss_factorization* f, T* x, int64_t N, int nrhs, cudaStream_t st, T* topz) {
  if (f->ntop <= 0) return RSS_OK;
  const unsigned nz = cdiv(nrhs, RC);
  const size_t tsm = sizeof(T) * (size_t)f->ntop * RC;
  if (tsm > 200 * 1024) {
    rss_set_error("rss_solve: top block too large for the on-chip solve");
    return RSS_EINVAL;
  }
  RSS_CUDA(cudaFuncSetAttribute(k_top_gemv<T, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  const unsigned g = std::min<long long>(cdiv((long long)f->ntop * nz * RC, 256), 152LL * 8);
  k_top_gather<T><<<g, 256, 0, st>>>(f->d_top_idx, f->ntop, x, N, nrhs, topz);
  RSS_LAUNCHED();
  k_top_gemv<T, RC><<<dim3(cdiv(f->ntop, SW_NT), nz), SW_NT, tsm, st>>>(static_cast<const T*>(f->d_top_inv),
                                                                        f->d_top_idx, f->ntop, topz, x, N, nrhs);
  RSS_LAUNCHED();
  return RSS_OK;
}

// The two persistent launches of the FP64 sweeps (k_sweep) around the top
// block.  Shared memory: the most any class needs without staging its small
// matrices (at least 48 KB; more room lets them be staged); the grid: as many
// CTAs as fit on the device at once (a cooperative launch needs all of them
// resident).  *done is false when the launch is not possible (the caller then
// takes the per-class kernels).
constexpr long long SWP_POLLS = 1LL << 24;

template <typename T, int RC> size_t sweep_persistent_smem(const rss_factorization* f, int k0) {
  size_t need = 0;
  for (size_t i = k0; i < f->batches.size(); ++i) {
    const Batch& b = f->batches[i];
    const size_t up = (size_t)(b.max_k + 2 * b.max_r + SW_SUB_U * b.max_r) * RC;
    const size_t dn = (size_t)b.max_r * RC + swp_dn_part_sm(b.max_r, RC);
    const size_t fin = (size_t)(3 * b.max_r + SW_SUB_T * std::max(b.max_r, b.max_k)) * RC;
    need = std::max(need, std::max(up, std::max(dn, fin)));
  }
  const size_t smem = std::max(need * sizeof(T), size_t(16) << 10);
  return (smem + 1023) & ~size_t(1023);
}

// One persistent launch (k_sweep) over the colour classes k0 .. end of the
// factor order: upward in that order, or downward in reverse.
template <typename T, int RC>
rss_status sweep_persistent_launch(const rss_factorization* f, T* x, int64_t N, int nrhs, cudaStream_t st,
                                   T* part, unsigned* bar, int k0, bool up) {
  const size_t smem = sweep_persistent_smem<T, RC>(f, k0);
  int dev = 0, sms = 0;
  RSS_CUDA(cudaGetDevice(&dev));
  RSS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SwpArgs<T> a;
  a.cls = static_cast<const SwpClass<T>*>(f->d_swp) + k0;
  a.ncls = (int)f->batches.size() - k0;
  a.x = x;
  a.N = N;
  a.nrhs = nrhs;
  a.part = part;
  a.bar = bar;
  a.err = reinterpret_cast<int*>(bar + 2);
  a.polls = f->params.wait_polls == 0 ? SWP_POLLS : f->params.wait_polls < 0 ? 0 : (long long)f->params.wait_polls;
  a.sm_cap = (int)(smem / sizeof(T));
  a.spread = f->swp_spread > 0 ? f->swp_spread : SWP_SPREAD_DEFAULT;
  void* args[] = {&a};
  const void* fn = up ? reinterpret_cast<const void*>(k_sweep<T, RC, true>)
                      : reinterpret_cast<const void*>(k_sweep<T, RC, false>);
  RSS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  RSS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, SWP_NT, smem));
  if (per_sm < 1) {
    rss_set_error("rss_solve: the persistent sweep kernel does not fit an SM");
    return RSS_ECUDA;
  }
  if (f->swp_ctas > 0) per_sm = std::min(per_sm, f->swp_ctas);
  RSS_CUDA(cudaLaunchCooperativeKernel(fn, dim3(per_sm * sms), dim3(SWP_NT), args, smem, st));
  return RSS_OK;
}

// First colour class of the persistent part of the sweeps: the whole factor
// (form 2), the tail of classes with fewer than f->swp_tail_boxes boxes each
// (form 3), or none (per-class kernels; also when the device or the factor's
// box sizes do not allow the cooperative launch).
template <typename T, int RC> int sweep_persistent_start(const rss_factorization* f) {
  const int nb = (int)f->batches.size();
  if (!f->d_swp || nb == 0 || (f->swp_launch != 2 && f->swp_launch != 3)) return nb;
  int k0 = 0;
  if (f->swp_launch == 3) {
    k0 = nb;
    while (k0 > 0 && f->batches[k0 - 1].nrec < f->swp_tail_boxes) --k0;
  }
  if (k0 == nb || sweep_persistent_smem<T, RC>(f, k0) > (size_t(200) << 10)) return nb;
  int dev = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
    cudaGetLastError();
    return nb;
  }
  return k0;
}

// tcz: complex factors with at least ZCN right-hand sides take the tensor-core
// sweeps (k_up_tcz, k_down_tcz) for every colour class whose boxes fit their
// shared memory and that gives at least one CTA per SM (boxes x column chunks);
// smaller classes, whose one-CTA-per-box chain of products would be latency
// bound, keep these FP64 kernels, which spread the rows of C over CTAs.
template <typename T, int RC>
rss_status sweeps(const rss_factorization* f, T* x, int64_t N, int nrhs, cudaStream_t st, void* ws,
                  bool tcz = false) {
  const unsigned nz = cdiv(nrhs, RC);
  const unsigned nzc = cdiv(nrhs, ZCN);
  if constexpr (std::is_same<T, zd>::value) {
    if (tcz) {
      RSS_CUDA(cudaFuncSetAttribute(k_up_tcz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TCZ_SMEM_MAX));
      RSS_CUDA(cudaFuncSetAttribute(k_down_tcz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TCZ_SMEM_MAX));
    }
  }
  const SweepWs w = sweep_ws<T>(f, nrhs, RC);
  char* wb = static_cast<char*>(ws);
  T* part = reinterpret_cast<T*>(wb);
  int* cnt = reinterpret_cast<int*>(wb + w.cnt_off);
  T* topz = reinterpret_cast<T*>(wb + w.topz_off);
  RSS_CUDA(cudaMemsetAsync(cnt, 0, w.topz_off - w.cnt_off, st));
  // classes k0 .. end go through the persistent launches (none, all, or the
  // coarse tail), the others through the per-class kernels
  const int nb = (int)f->batches.size();
  const int k0 = tcz ? nb : sweep_persistent_start<T, RC>(f);
  unsigned* bar = reinterpret_cast<unsigned*>(wb + w.bar_off);
  RSS_CUDA(cudaFuncSetAttribute(k_up_r<T, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  RSS_CUDA(cudaFuncSetAttribute(k_up_c<T, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  RSS_CUDA(cudaFuncSetAttribute(k_down<T, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  RSS_CUDA(cudaFuncSetAttribute(k_top_gemv<T, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  for (int bi = 0; bi < k0; ++bi) {
    const Batch& b = f->batches[bi];
    const BoxRec<T>* recs = static_cast<const BoxRec<T>*>(b.d_recs);
    if constexpr (std::is_same<T, zd>::value) {
      const size_t sm = tcz_smem_up(b.max_k, b.max_r);
      if (tcz && sm <= TCZ_SMEM_MAX && (long long)b.nrec * nzc >= 152) {
        k_up_tcz<<<dim3(b.nrec, nzc), TC_NT, sm, st>>>(recs, x, N, nrhs);
        RSS_LAUNCHED();
        continue;
      }
    }
    const size_t need_r = sizeof(T) * (size_t)(b.max_k + b.max_r + SW_SUB_U * b.max_r) * RC;
    const size_t want_r = need_r + sizeof(T) * ((size_t)(b.max_k | 1) * b.max_r + (size_t)b.max_r * b.max_r);
    const size_t sm_r = std::max(std::min<size_t>(want_r, 96 * 1024), need_r);
    if (sm_r > 200 * 1024) {
      rss_set_error("rss_solve: a box's upward sweep needs more shared memory than an SM has");
      return RSS_EINVAL;
    }
    k_up_r<T, RC><<<dim3(b.nrec, 1, nz), SW_NT_U, sm_r, st>>>(recs, x, N, nrhs, (int)(sm_r / sizeof(T)));
    RSS_LAUNCHED();
    k_up_c<T, RC><<<dim3(cdiv(b.max_c, SW_ROWS), b.nrec, nz), SW_NT, sizeof(T) * (size_t)b.max_r * RC, st>>>(
        recs, x, N, nrhs);
    RSS_LAUNCHED();
  }
  if (k0 < nb) {
    const rss_status sp = sweep_persistent_launch<T, RC>(f, x, N, nrhs, st, part, bar, k0, true);
    if (sp != RSS_OK) return sp;
  }
  {
    const rss_status stp = top_apply<T, RC>(f, x, N, nrhs, st, topz);
    if (stp != RSS_OK) return stp;
  }
  if (k0 < nb) {
    const rss_status sp = sweep_persistent_launch<T, RC>(f, x, N, nrhs, st, part, bar, k0, false);
    if (sp != RSS_OK) return sp;
  }
  for (int bi = k0 - 1; bi >= 0; --bi) {
    const Batch* it = &f->batches[bi];
    if constexpr (std::is_same<T, zd>::value) {
      const size_t sm = tcz_smem_down(it->max_r);
      if (tcz && tcz_smem_up(it->max_k, it->max_r) <= TCZ_SMEM_MAX &&
          (long long)it->nrec * nzc >= 152) {   // the same classes as upward
        k_down_tcz<<<dim3(it->nrec, nzc), TC_NT, sm, st>>>(static_cast<const BoxRec<T>*>(it->d_recs), x, N, nrhs);
        RSS_LAUNCHED();
        continue;
      }
    }
    {   // classes with many boxes: one CTA per box, no partial sums through global memory
      const size_t need_b = sizeof(T) * down_box_sm<T, RC>(it->max_r, it->max_k);
      if ((long long)it->nrec * nz >= 2 * 152 && need_b <= 96 * 1024) {
        const size_t want_b = sizeof(T) * ((size_t)(3 * it->max_r + SW_SUB_T * std::max(it->max_r, it->max_k)) * RC +
                                           (size_t)it->max_r * it->max_r + (size_t)(it->max_k | 1) * it->max_r);
        const size_t sm_b = std::max(need_b, std::min<size_t>(want_b, 96 * 1024));
        RSS_CUDA(cudaFuncSetAttribute(k_down_box<T, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_b));
        k_down_box<T, RC><<<dim3(it->nrec, 1, nz), SW_NT_D, sm_b, st>>>(static_cast<const BoxRec<T>*>(it->d_recs), x,
                                                                       N, nrhs, (int)(sm_b / sizeof(T)));
        RSS_LAUNCHED();
        continue;
      }
    }
    const int nch = (int)cdiv(it->max_c, SW_ROWS_D);
    const size_t want_d =
        sizeof(T) * std::max((size_t)SW_ROWS_D * RC + (size_t)SW_SUB_D * it->max_r * RC +
                                 (size_t)(SW_ROWS_D + 1) * it->max_r,
                             (size_t)(2 * it->max_r + SW_SUB_T * std::max(it->max_r, it->max_k)) * RC +
                                 (size_t)it->max_r * it->max_r + (size_t)(it->max_k | 1) * it->max_r);
    // y_C and the parts' sums (and later z, y_R) are always in shared memory; the
    // staged blocks only when they fit
    const size_t need_d =
        sizeof(T) * std::max((size_t)SW_ROWS_D * RC + (size_t)SW_SUB_D * it->max_r * RC,
                             (size_t)(2 * it->max_r + SW_SUB_T * std::max(it->max_r, it->max_k)) * RC);
    const size_t sm_d = std::max(std::min<size_t>(want_d, 96 * 1024), need_d);
    if (sm_d > 200 * 1024) {
      rss_set_error("rss_solve: a box's downward sweep needs more shared memory than an SM has");
      return RSS_EINVAL;
    }
    k_down<T, RC><<<dim3(nch, it->nrec, nz), SW_NT_D, sm_d, st>>>(static_cast<const BoxRec<T>*>(it->d_recs), x, N,
                                                                nrhs, part, cnt, nch, it->max_r, (int)(sm_d / sizeof(T)));
    RSS_LAUNCHED();
  }
  return RSS_OK;
}

// The digit slices of E and F for the tensor-core sweeps: built once per factor
// by the first solve that needs them (on its stream, which it then waits for),
// kept until the factor is freed.  Boxes with c >= 1024 keep the per-chunk
// products (the int64 sums of tc_gemm_sl need K < 1024).
bool slices_fit(const rss_factorization* f) {
  for (const Batch& b : f->batches)
    if (b.max_c >= 1024) return false;
  return true;
}

size_t slice_total(const rss_factorization* f) {
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  size_t total = 0;
  for (size_t bi = 0; bi < f->batches.size(); ++bi) {
    const Batch& b = f->batches[bi];
    const BoxRec<double>* hr = static_cast<const BoxRec<double>*>(f->rec_host[bi]);
    total += al(sizeof(SliceRec) * b.nrec);
    for (int q = 0; q < b.nrec; ++q) {
      const size_t kp = (hr[q].r + 15) & ~15, cp = (hr[q].c + 15) & ~15;
      total += al(sizeof(uint16_t) * hr[q].c * OZ_S * kp) + al(sizeof(int) * hr[q].c) +
               al(sizeof(uint16_t) * hr[q].r * OZ_S * cp) + al(sizeof(int) * hr[q].r);
    }
  }
  return total;
}

rss_status ensure_slices(rss_factorization* f, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(f->slice_mu);
  if (f->slices_ready) return RSS_OK;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t total = slice_total(f);
  char* base = nullptr;
  RSS_CUDA(pool_malloc(reinterpret_cast<void**>(&base), total, st));
  char* p = base;
  auto take = [&](size_t b) {
    char* q = p;
    p += al(b);
    return q;
  };
  std::vector<SliceRec*> recs(f->batches.size());
  std::vector<SliceRec> hs;
  for (size_t bi = 0; bi < f->batches.size(); ++bi) {
    const Batch& b = f->batches[bi];
    const BoxRec<double>* hr = static_cast<const BoxRec<double>*>(f->rec_host[bi]);
    recs[bi] = reinterpret_cast<SliceRec*>(take(sizeof(SliceRec) * b.nrec));
    hs.assign(b.nrec, SliceRec{});
    for (int q = 0; q < b.nrec; ++q) {
      SliceRec& S = hs[q];
      S.kp = (hr[q].r + 15) & ~15;
      S.cp = (hr[q].c + 15) & ~15;
      S.Esl = reinterpret_cast<uint16_t*>(take(sizeof(uint16_t) * hr[q].c * OZ_S * S.kp));
      S.Eexp = reinterpret_cast<int*>(take(sizeof(int) * hr[q].c));
      S.Fsl = reinterpret_cast<uint16_t*>(take(sizeof(uint16_t) * hr[q].r * OZ_S * S.cp));
      S.Fexp = reinterpret_cast<int*>(take(sizeof(int) * hr[q].r));
    }
    cudaError_t e = cudaMemcpyAsync(recs[bi], hs.data(), sizeof(SliceRec) * b.nrec, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // hs is reused for the next batch
    if (e == cudaSuccess) {
      const BoxRec<double>* dr = static_cast<const BoxRec<double>*>(b.d_recs);
      k_slice_e<<<dim3(b.nrec, cdiv(b.max_c, 64)), TC_NT, 0, st>>>(dr, recs[bi]);
      k_slice_f<<<dim3(b.nrec, cdiv(b.max_r, TC_NT / 32)), TC_NT, 0, st>>>(dr, recs[bi]);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
      cudaStreamSynchronize(st);
      pool_free(base, st);
      rss_set_error(std::string("rss_solve: slice cache: ") + cudaGetErrorString(e));
      return RSS_ECUDA;
    }
  }
  RSS_CUDA(cudaStreamSynchronize(st));   // other streams may use the slices from here on
  f->slice_bytes = total;
  f->d_slice_mem = base;
  f->d_slices = recs;
  f->slices_ready = true;
  return RSS_OK;
}

// Real factors with at least TCN right-hand sides: the tensor-core sweeps; the
// top block as in sweeps<double, 8>.
// may_build: the caller allows the one-time allocation of the slice cache
// (rss_solve_noalloc does not; it uses the cache only when it already exists).
rss_status sweeps_tc(const rss_factorization* f, double* x, int64_t N, int nrhs, cudaStream_t st, void* ws,
                     bool may_build) {
  constexpr int RC = 8;
  bool sl = slices_fit(f);
  if (sl && may_build) {
    const rss_status s = ensure_slices(const_cast<rss_factorization*>(f), st);
    if (s != RSS_OK) return s;
  } else if (sl) {
    std::lock_guard<std::mutex> lk(const_cast<rss_factorization*>(f)->slice_mu);
    sl = f->slices_ready;
  }
  const unsigned nz = cdiv(nrhs, TCN);
  const SweepWs w = sweep_ws<double>(f, nrhs, RC);
  double* topz = reinterpret_cast<double*>(static_cast<char*>(ws) + w.topz_off);
  RSS_CUDA(cudaFuncSetAttribute(k_up_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
  RSS_CUDA(cudaFuncSetAttribute(k_down_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
  RSS_CUDA(cudaFuncSetAttribute(k_top_gemv<double, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  const size_t head = (size_t)(TCM + TCN) * TSA * sizeof(uint16_t);
  for (size_t bi = 0; bi < f->batches.size(); ++bi) {
    const Batch& b = f->batches[bi];
    const size_t sm = head + sizeof(double) * (size_t)(b.max_k + 2 * b.max_r) * TCN;
    if (sm > 220 * 1024) {
      rss_set_error("rss_solve: box too large for the tensor-core sweep");
      return RSS_EINVAL;
    }
    k_up_tc<<<dim3(b.nrec, nz), TC_NT, sm, st>>>(static_cast<const BoxRec<double>*>(b.d_recs),
                                                  sl ? f->d_slices[bi] : nullptr, x, N, nrhs);
    RSS_LAUNCHED();
  }
  if (f->ntop > 0) {
    const unsigned nz8 = cdiv(nrhs, RC);
    const size_t tsm = sizeof(double) * (size_t)f->ntop * RC;
    if (tsm > 200 * 1024) {
      rss_set_error("rss_solve: top block too large for the on-chip solve");
      return RSS_EINVAL;
    }
    const unsigned g = std::min<long long>(cdiv((long long)f->ntop * nz8 * RC, 256), 152LL * 8);
    k_top_gather<double><<<g, 256, 0, st>>>(f->d_top_idx, f->ntop, x, N, nrhs, topz);
    RSS_LAUNCHED();
    k_top_gemv<double, RC><<<dim3(cdiv(f->ntop, SW_NT), nz8), SW_NT, tsm, st>>>(
        static_cast<const double*>(f->d_top_inv), f->d_top_idx, f->ntop, topz, x, N, nrhs);
    RSS_LAUNCHED();
  }
  for (size_t bi = f->batches.size(); bi-- > 0;) {
    const Batch& b = f->batches[bi];
    const size_t sm = head + sizeof(double) * (size_t)(2 * b.max_r) * TCN;
    k_down_tc<<<dim3(b.nrec, nz), TC_NT, sm, st>>>(static_cast<const BoxRec<double>*>(b.d_recs),
                                                    sl ? f->d_slices[bi] : nullptr, x, N, nrhs);
    RSS_LAUNCHED();
  }
  return RSS_OK;
}

bool use_tc(const rss_factorization* f, int64_t nrhs) {
  return !f->is_complex && nrhs >= TCN && (f->params.schur_path == 0 || f->params.schur_path == 2);
}

template <typename T>
rss_status run_sweeps(const rss_factorization* f, T* x, int64_t N, int64_t nrhs, cudaStream_t st, void* ws,
                      bool may_build = true) {
  if constexpr (sizeof(T) == sizeof(double))
    if (use_tc(f, nrhs)) return sweeps_tc(f, x, N, (int)nrhs, st, ws, may_build);
  const int rc = rhs_chunk(nrhs);
  const bool tcz = f->is_complex && nrhs >= ZCN && (f->params.schur_path == 0 || f->params.schur_path == 2);
  return rc == 1 ? sweeps<T, 1>(f, x, N, (int)nrhs, st, ws, tcz)
         : rc == 4 ? sweeps<T, 4>(f, x, N, (int)nrhs, st, ws, tcz)
                   : sweeps<T, 8>(f, x, N, (int)nrhs, st, ws, tcz);
}

}  // namespace

// A_top^{-1}, column by column from the LU (identity right-hand sides).
template <typename T> rss_status top_inverse(const T* LU, const int* piv, int n, T* Ainv, cudaStream_t st) {
  constexpr int RT = 4;
  const size_t tsm = sizeof(T) * (size_t)n * RT;
  if (tsm > 200 * 1024) {
    rss_set_error("rss_factor: top block too large for the on-chip solve");
    return RSS_EINVAL;
  }
  int* iota = nullptr;
  RSS_CUDA(pool_malloc(reinterpret_cast<void**>(&iota), sizeof(int) * (size_t)n, st));
  k_iota<<<cdiv(n, 256), 256, 0, st>>>(iota, n);
  k_identity<T><<<std::min<long long>(cdiv((long long)n * n, 256), 152LL * 8), 256, 0, st>>>(Ainv, n);
  RSS_CUDA(cudaFuncSetAttribute(k_top_solve<T, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  k_top_solve<T, RT><<<cdiv(n, RT), 1024, tsm, st>>>(LU, piv, iota, n, Ainv, n, n);
  const cudaError_t e = cudaGetLastError();
  pool_free(iota, st);
  if (e != cudaSuccess) {
    rss_set_error(std::string("rss_factor: top inverse launch failed: ") + cudaGetErrorString(e));
    return RSS_ECUDA;
  }
  return RSS_OK;
}

template rss_status top_inverse<double>(const double*, const int*, int, double*, cudaStream_t);
template rss_status top_inverse<zd>(const zd*, const int*, int, zd*, cudaStream_t);

template <typename T>
rss_status solve_impl(const rss_factorization* f, T* b, int64_t nrhs, int64_t ldb, cudaStream_t st) {
  const int64_t N = f->n;
  const SweepWs w = sweep_ws<T>(f, nrhs, rhs_chunk(nrhs));
  const size_t xb = (sizeof(T) * (size_t)N * nrhs + 255) & ~size_t(255);
  char* mem = nullptr;
  RSS_CUDA(pool_malloc(reinterpret_cast<void**>(&mem), xb + w.bytes, st));
  T* x = reinterpret_cast<T*>(mem);
  const int* err = reinterpret_cast<const int*>(mem + xb + w.bar_off + 2 * sizeof(unsigned));
  RSS_CUDA(cudaMemsetAsync(mem + xb + w.bar_off, 0, 4 * sizeof(int), st));
  const unsigned grid = std::min<long long>(cdiv((long long)N * nrhs, NT), 152LL * 16);
  k_perm_in<T><<<grid, NT, 0, st>>>(b, ldb, x, N, (int)nrhs, f->d_user_to_tree);
  rss_status s = RSS_OK;
  if (cudaGetLastError() != cudaSuccess) {
    rss_set_error("rss_solve: launch failed");
    s = RSS_ECUDA;
  }
  if (s == RSS_OK) s = run_sweeps<T>(f, x, N, nrhs, st, mem + xb);
  if (s == RSS_OK) {
    k_perm_out<T><<<grid, NT, 0, st>>>(b, ldb, x, N, (int)nrhs, f->d_user_to_tree, err);
    if (cudaGetLastError() != cudaSuccess) {
      rss_set_error("rss_solve: launch failed");
      s = RSS_ECUDA;
    }
  }
  pool_free(mem, st);
  return s;
}

template rss_status solve_impl<double>(const rss_factorization*, double*, int64_t, int64_t, cudaStream_t);

template <typename T> rss_status build_sweep_classes(rss_factorization* f, cudaStream_t st) {
  if (f->batches.empty()) return RSS_OK;
  std::vector<SwpClass<T>> h(f->batches.size());
  for (size_t i = 0; i < h.size(); ++i) {
    const Batch& b = f->batches[i];
    h[i] = SwpClass<T>{static_cast<const BoxRec<T>*>(b.d_recs), b.nrec, b.max_k, b.max_r, b.max_c};
  }
  void* d = f->arena.get(sizeof(SwpClass<T>) * h.size());
  if (!d) {
    rss_set_error("rss_factor: device arena allocation failed");
    return RSS_ENOMEM;
  }
  RSS_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(SwpClass<T>) * h.size(), cudaMemcpyHostToDevice, st));
  RSS_CUDA(cudaStreamSynchronize(st));   // h is a host temporary
  f->d_swp = d;
  return RSS_OK;
}

template rss_status build_sweep_classes<double>(rss_factorization*, cudaStream_t);
template rss_status build_sweep_classes<zd>(rss_factorization*, cudaStream_t);

size_t solve_device_bytes(const rss_factorization* f, int64_t nrhs) {
  const size_t esz = f->is_complex ? 16 : 8;
  const size_t xb = (esz * (size_t)f->n * (size_t)nrhs + 255) & ~size_t(255);
  return xb + (f->is_complex ? sweep_ws<zd>(f, nrhs, rhs_chunk(nrhs)).bytes
                             : sweep_ws<double>(f, nrhs, rhs_chunk(nrhs)).bytes);
}

size_t solve_cache_bytes(const rss_factorization* f, int64_t max_nrhs) {
  return use_tc(f, max_nrhs) && slices_fit(f) ? slice_total(f) : 0;
}

rss_status prepare_solve_caches(const rss_factorization* f, int64_t max_nrhs, cudaStream_t st) {
  if (!use_tc(f, max_nrhs) || !slices_fit(f)) return RSS_OK;
  return ensure_slices(const_cast<rss_factorization*>(f), st);
}
template rss_status solve_impl<zd>(const rss_factorization*, zd*, int64_t, int64_t, cudaStream_t);

// ---------------------------------------------------------------------------
// rss_solve_noalloc: the same sweeps as rss_solve, with the working copy of
// the right-hand sides in a fixed device array instead of memory obtained at
// call time.  Some callers cannot allocate device memory: a process whose
// framework allocator has already reserved the device's free memory, a
// latency-bound serving loop that may not take the synchronisation a fresh
// allocation can cost, or a host that budgets device memory up front.  For
// them the scratch is a file-scope array that exists on every GPU that loads
// the library, for the life of the process.

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the symbol's host-side name is not a device address).
rss_status noalloc_scratch(void** out) {
  int dev = -1;
  RSS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    rss_set_error("rss_solve_noalloc: device ordinal out of range");
    return RSS_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    RSS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return RSS_OK;
}

template <typename T>
rss_status solve_in_scratch(const rss_factorization* f, T* b, int64_t nrhs, int64_t ldb, cudaStream_t st,
                            T* x) {
  const int64_t N = f->n;
  const unsigned grid = std::min<long long>(cdiv((long long)N * nrhs, NT), 152LL * 16);
  // every entry of x is written here, so nothing left from an earlier call is read
  k_perm_in<T><<<grid, NT, 0, st>>>(b, ldb, x, N, (int)nrhs, f->d_user_to_tree);
  RSS_LAUNCHED();
  const size_t xb = (sizeof(T) * (size_t)N * nrhs + 255) & ~size_t(255);
  char* ws = reinterpret_cast<char*>(x) + xb;
  const SweepWs w = sweep_ws<T>(f, nrhs, rhs_chunk(nrhs));
  RSS_CUDA(cudaMemsetAsync(ws + w.bar_off, 0, 4 * sizeof(int), st));   // barrier words of the last call
  const rss_status s = run_sweeps<T>(f, x, N, nrhs, st, ws, false);
  if (s != RSS_OK) return s;
  k_perm_out<T><<<grid, NT, 0, st>>>(b, ldb, x, N, (int)nrhs, f->d_user_to_tree,
                                     reinterpret_cast<const int*>(ws + w.bar_off + 2 * sizeof(unsigned)));
  RSS_LAUNCHED();
  return RSS_OK;
}

}  // namespace

extern "C" rss_status rss_solve_noalloc(const rss_factorization* f, void* b, int64_t nrhs, int64_t ldb,
                                        void* stream) {
  if (!f || f->tag != RSS_TAG_FACTOR) {
    rss_set_error("rss_solve_noalloc: not a factor handle");
    return RSS_EINVAL;
  }
  if (!b || nrhs <= 0 || ldb < f->n) {
    rss_set_error("rss_solve_noalloc: b must be non-NULL with nrhs > 0 and ldb >= n");
    return RSS_EINVAL;
  }
  const size_t esz = f->is_complex ? 16 : 8;
  const size_t need = ((esz * (size_t)f->n * (size_t)nrhs + 255) & ~size_t(255)) +
                      (f->is_complex ? sweep_ws<zd>(f, nrhs, rhs_chunk(nrhs)).bytes
                                     : sweep_ws<double>(f, nrhs, rhs_chunk(nrhs)).bytes);
  if (need > kNoAllocScratchBytes) {
    rss_set_error("rss_solve_noalloc: n * nrhs (with the sweep workspace) needs " + std::to_string(need) +
                  " bytes of scratch; the fixed maximum is " + std::to_string(kNoAllocScratchBytes) +
                  " bytes (use rss_solve, or fewer right-hand sides per call)");
    return RSS_EINVAL;
  }
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, b) != cudaSuccess) {
    cudaGetLastError();
    attr.type = cudaMemoryTypeUnregistered;
  }
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) {
    rss_set_error("rss_solve_noalloc: b must be device memory (staging host data would allocate)");
    return RSS_EINVAL;
  }
  void* scratch = nullptr;
  rss_status s = noalloc_scratch(&scratch);
  if (s != RSS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return f->is_complex
             ? solve_in_scratch<zd>(f, static_cast<zd*>(b), nrhs, ldb, st, static_cast<zd*>(scratch))
             : solve_in_scratch<double>(f, static_cast<double*>(b), nrhs, ldb, st, static_cast<double*>(scratch));
}

// ---------------------------------------------------------------------------
// rss_tune_solve: the schedule of the persistent sweeps, chosen by measurement.
// The knob is `spread`, the target number of work items per CTA and colour
// class: 1 keeps whole boxes per CTA wherever a class has about as many boxes
// as the GPU has CTAs, larger values split the boxes of more classes into
// groups of 64-row chunks of C (more parallel work, one more grid barrier per
// split class).  Every schedule adds the same products in the same order, so
// the choice changes the time of a solve, never its result.
extern "C" rss_status rss_tune_solve(rss_factorization* f, int64_t nrhs, void* stream, char* json, size_t len) {
  if (!f || f->tag != RSS_TAG_FACTOR || nrhs <= 0 || nrhs >= 1 << 20) {
    rss_set_error("rss_tune_solve: needs a factor handle and 0 < nrhs < 2^20");
    return RSS_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t esz = f->is_complex ? 16 : 8;
  const bool fp64_path = f->is_complex ? nrhs < ZCN : !use_tc(f, nrhs);
  std::ostringstream o;
  o << "{\"nrhs\": " << nrhs;
  if (!fp64_path || !f->d_swp) {
    o << ", \"path\": \"tensor-core sweeps (nothing to tune)\"}";
  } else {
    const size_t bytes = esz * (size_t)f->n * (size_t)nrhs;
    void* b = nullptr;
    RSS_CUDA(pool_malloc(&b, bytes, st));
    RSS_CUDA(cudaMemsetAsync(b, 0, bytes, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    RSS_CUDA(cudaEventCreate(&e0));
    RSS_CUDA(cudaEventCreate(&e1));
    struct Cand {
      int launch, spread, ctas, tail;
    };
    const Cand cands[] = {{1, 0, 0, 0},   {2, 1, 4, 0},   {2, 1, 0, 0},   {2, 4, 4, 0},
                          {2, 4, 0, 0},   {3, 1, 0, 32},  {3, 4, 0, 32},  {3, 1, 0, 128},
                          {3, 4, 0, 128}, {3, 1, 0, 512}, {3, 4, 0, 512}};
    const int ncand = (int)(sizeof(cands) / sizeof(cands[0]));
    const int keep = f->swp_spread, keep_c = f->swp_ctas, keep_l = f->swp_launch, keep_t = f->swp_tail_boxes;
    Cand best{1, 0, 0, 0};
    float best_ms = 1e30f;
    rss_status s = RSS_OK;
    o << ", \"path\": \"FP64 sweeps\", \"candidates\": [";
    for (int ci = 0; ci < ncand && s == RSS_OK; ++ci) {
      const Cand& c = cands[ci];
      f->swp_launch = c.launch;
      f->swp_spread = c.spread;
      f->swp_ctas = c.ctas;
      f->swp_tail_boxes = c.tail;
      float t[3];
      for (int rep = -1; rep < 3 && s == RSS_OK; ++rep) {   // one untimed run first
        cudaEventRecord(e0, st);
        s = f->is_complex ? solve_impl<zd>(f, static_cast<zd*>(b), nrhs, f->n, st)
                          : solve_impl<double>(f, static_cast<double*>(b), nrhs, f->n, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) s = RSS_ECUDA;
        if (rep >= 0 && s == RSS_OK) cudaEventElapsedTime(&t[rep], e0, e1);
      }
      if (s != RSS_OK) break;
      std::sort(t, t + 3);
      o << (ci ? ", " : "") << "{\"launch\": \"" << (c.launch == 1 ? "per_class" : c.launch == 2 ? "persistent" : "hybrid")
        << "\"";
      if (c.launch != 1) o << ", \"spread\": " << c.spread << ", \"ctas_per_sm\": " << c.ctas;
      if (c.launch == 3) o << ", \"tail_boxes\": " << c.tail;
      o << ", \"ms\": " << t[1] << "}";
      if (t[1] < best_ms) {
        best_ms = t[1];
        best = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pool_free(b, st);
    if (s != RSS_OK) {
      f->swp_spread = keep;
      f->swp_ctas = keep_c;
      f->swp_launch = keep_l;
      f->swp_tail_boxes = keep_t;
      return s;
    }
    f->swp_launch = best.launch;
    f->swp_spread = best.spread;
    f->swp_ctas = best.ctas;
    f->swp_tail_boxes = best.tail;
    o << "], \"launch\": \"" << (best.launch == 1 ? "per_class" : best.launch == 2 ? "persistent" : "hybrid")
      << "\"";
    if (best.launch != 1) o << ", \"spread\": " << best.spread << ", \"ctas_per_sm\": " << best.ctas;
    if (best.launch == 3) o << ", \"tail_boxes\": " << best.tail;
    o << ", \"ms\": " << best_ms << "}";
  }
  const std::string js = o.str();
  if (json && len) {
    if (js.size() + 1 > len) {
      rss_set_error("rss_tune_solve: json buffer too small");
      return RSS_EINVAL;
    }
    std::memcpy(json, js.c_str(), js.size() + 1);
  }
  return RSS_OK;
}
