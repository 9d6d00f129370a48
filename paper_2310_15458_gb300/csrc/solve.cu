// Applying the factorization (Section 2.5): x = W_1 .. W_K A_top^{-1} V_K .. V_1 b.
//
// Upward sweep, boxes in factor order (each colour class in one launch):
//   b_R -= T^* b_S;  b_R <- L_R^{-1} P_R b_R;  b_C -= E b_R          (apply V)
// dense top solve, then the downward sweep in reverse order:
//   y_R <- U_R^{-1} (y_R - F y_C);  y_S -= T y_R                       (apply W)
// Boxes of one colour class touch disjoint entries of x, so a class is one
// launch; the right-hand sides are split into chunks of RC columns.
#include <algorithm>
#include <mutex>

#include "internal.h"

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
                           const int* __restrict__ u2t) {
  const long long tot = (long long)N * nrhs;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e % N, j = e / N;
    b[i + j * ldb] = x[u2t[i] + j * N];
  }
}

template <typename T, int RC>
__global__ void __launch_bounds__(NT) k_solve_up(const BoxRec<T>* __restrict__ recs, T* __restrict__ x, int64_t N,
                                                 int nrhs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BoxRec<T> R = recs[blockIdx.x];
  const int k = R.k, r = R.r, c = R.c;
  const int q0 = blockIdx.y * RC, nq = min(RC, nrhs - q0);
  T* bS = reinterpret_cast<T*>(smraw);   // k x RC
  T* t = bS + (size_t)k * RC;            // r x RC
  T* bR = t + (size_t)r * RC;            // r x RC
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
  __syncthreads();
  for (int e = tid; e < r * RC; e += bs) {        // b_R - T^* b_S
    const int j = e / RC, q = e % RC;
    T acc = t[e];
    for (int s = 0; s < k; ++s) acc = msbc(acc, R.Tm[s + (size_t)j * k], bS[s * RC + q]);
    t[e] = acc;
  }
  __syncthreads();
  for (int e = tid; e < r * RC; e += bs) {        // L_R^{-1} P_R (b_R - T^* b_S)
    const int j = e / RC, q = e % RC;
    T acc = zero<T>();
    for (int l = 0; l < r; ++l) acc = mad(acc, R.LiP[j + (size_t)l * r], t[l * RC + q]);
    bR[e] = acc;
    if (q < nq) xq[R.idxR[j] + (int64_t)q * N] = acc;
  }
  __syncthreads();
  for (int i = tid; i < c; i += bs) {             // b_C -= E b_R
    T acc[RC];
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = zero<T>();
    for (int j = 0; j < r; ++j) {
      const T e = R.E[i + (size_t)j * c];
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = mad(acc[q], e, bR[j * RC + q]);
    }
    const int gi = R.idxC[i];
#pragma unroll
    for (int q = 0; q < RC; ++q)
      if (q < nq) xq[gi + (int64_t)q * N] = xq[gi + (int64_t)q * N] - acc[q];
  }
}

template <typename T, int RC>
__global__ void __launch_bounds__(NT) k_solve_down(const BoxRec<T>* __restrict__ recs, T* __restrict__ x,
                                                   int64_t N, int nrhs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BoxRec<T> R = recs[blockIdx.x];
  const int k = R.k, r = R.r, c = R.c;
  const int q0 = blockIdx.y * RC, nq = min(RC, nrhs - q0);
  T* t = reinterpret_cast<T*>(smraw);   // r x RC
  T* yR = t + (size_t)r * RC;           // r x RC
  T* yC = yR + (size_t)r * RC;          // c x RC: y_C gathered once
  const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = bs >> 5;
  T* xq = x + (int64_t)q0 * N;
  for (int e = tid; e < c * RC; e += bs) {
    const int i = e / RC, q = e % RC;
    yC[e] = q < nq ? xq[R.idxC[i] + (int64_t)q * N] : zero<T>();
  }
  __syncthreads();
  for (int j = warp; j < r; j += nw) {            // y_R - F y_C
    T acc[RC];
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = zero<T>();
    for (int i = lane; i < c; i += 32) {
      const T fv = R.Ft[i + (size_t)j * c];
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = mad(acc[q], fv, yC[i * RC + q]);
    }
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = warp_sum(acc[q]);
    if (lane == 0) {
      const int gj = R.idxR[j];
#pragma unroll
      for (int q = 0; q < RC; ++q) t[j * RC + q] = q < nq ? xq[gj + (int64_t)q * N] - acc[q] : zero<T>();
    }
  }
  __syncthreads();
  for (int e = tid; e < r * RC; e += bs) {        // U_R^{-1} (y_R - F y_C)
    const int j = e / RC, q = e % RC;
    T acc = zero<T>();
    for (int l = j; l < r; ++l) acc = mad(acc, R.Ui[j + (size_t)l * r], t[l * RC + q]);
    yR[e] = acc;
    if (q < nq) xq[R.idxR[j] + (int64_t)q * N] = acc;
  }
  __syncthreads();
  for (int e = tid; e < k * RC; e += bs) {        // y_S -= T y_R
    const int s = e / RC, q = e % RC;
    if (q >= nq) continue;
    T acc = zero<T>();
    for (int j = 0; j < r; ++j) acc = mad(acc, R.Tm[s + (size_t)j * k], yR[j * RC + q]);
    const int gs = R.idxC[s];
    xq[gs + (int64_t)q * N] = xq[gs + (int64_t)q * N] - acc;
  }
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

template <typename T, int RC>
rss_status sweeps(const rss_factorization* f, T* x, int64_t N, int nrhs, cudaStream_t st) {
  const unsigned nchunk = cdiv(nrhs, RC);
  RSS_CUDA(cudaFuncSetAttribute(k_solve_up<T, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  RSS_CUDA(cudaFuncSetAttribute(k_solve_down<T, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  for (const Batch& b : f->batches) {
    const size_t smem = sizeof(T) * (size_t)(b.max_k + 2 * b.max_r) * RC;
    k_solve_up<T, RC><<<dim3(b.nrec, nchunk), NT, smem, st>>>(static_cast<const BoxRec<T>*>(b.d_recs), x, N, nrhs);
    RSS_LAUNCHED();
  }
  constexpr int RT = 4;
  const size_t tsm = sizeof(T) * (size_t)f->ntop * RT;
  if (tsm > 200 * 1024) {
    rss_set_error("rss_solve: top block too large for the on-chip solve");
    return RSS_EINVAL;
  }
  RSS_CUDA(cudaFuncSetAttribute(k_top_solve<T, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  if (f->ntop > 0) {
    k_top_solve<T, RT><<<cdiv(nrhs, RT), 1024, tsm, st>>>(static_cast<const T*>(f->d_top_lu), f->d_top_piv,
                                                         f->d_top_idx, f->ntop, x, N, nrhs);
    RSS_LAUNCHED();
  }
  for (auto it = f->batches.rbegin(); it != f->batches.rend(); ++it) {
    const size_t smem = sizeof(T) * (size_t)(2 * it->max_r + it->max_c) * RC;
    k_solve_down<T, RC><<<dim3(it->nrec, nchunk), NT, smem, st>>>(static_cast<const BoxRec<T>*>(it->d_recs), x, N,
                                                                 nrhs);
    RSS_LAUNCHED();
  }
  return RSS_OK;
}

}  // namespace

template <typename T>
rss_status solve_impl(const rss_factorization* f, T* b, int64_t nrhs, int64_t ldb, cudaStream_t st) {
  const int64_t N = f->n;
  T* x = nullptr;
  RSS_CUDA(cudaMallocAsync(&x, sizeof(T) * (size_t)N * nrhs, st));
  const unsigned grid = std::min<long long>(cdiv((long long)N * nrhs, NT), 152LL * 16);
  k_perm_in<T><<<grid, NT, 0, st>>>(b, ldb, x, N, (int)nrhs, f->d_user_to_tree);
  rss_status s = RSS_OK;
  if (cudaGetLastError() != cudaSuccess) {
    rss_set_error("rss_solve: launch failed");
    s = RSS_ECUDA;
  }
  if (s == RSS_OK) {
    if (nrhs == 1) s = sweeps<T, 1>(f, x, N, (int)nrhs, st);
    else if (nrhs <= 4) s = sweeps<T, 4>(f, x, N, (int)nrhs, st);
    else s = sweeps<T, 8>(f, x, N, (int)nrhs, st);
  }
  if (s == RSS_OK) {
    k_perm_out<T><<<grid, NT, 0, st>>>(b, ldb, x, N, (int)nrhs, f->d_user_to_tree);
    if (cudaGetLastError() != cudaSuccess) {
      rss_set_error("rss_solve: launch failed");
      s = RSS_ECUDA;
    }
  }
  cudaFreeAsync(x, st);
  return s;
}

template rss_status solve_impl<double>(const rss_factorization*, double*, int64_t, int64_t, cudaStream_t);
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
  rss_status s;
  if (nrhs == 1) s = sweeps<T, 1>(f, x, N, (int)nrhs, st);
  else if (nrhs <= 4) s = sweeps<T, 4>(f, x, N, (int)nrhs, st);
  else s = sweeps<T, 8>(f, x, N, (int)nrhs, st);
  if (s != RSS_OK) return s;
  k_perm_out<T><<<grid, NT, 0, st>>>(b, ldb, x, N, (int)nrhs, f->d_user_to_tree);
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
  const size_t need = esz * (size_t)f->n * (size_t)nrhs;
  if (need > kNoAllocScratchBytes) {
    rss_set_error("rss_solve_noalloc: n * nrhs needs " + std::to_string(need) +
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
