// The paper's discretisations and iterative refinement (Section 5).
//
//   self_integral        : integral of the kernel over one h x h cell (Eqs. 16, 20)
//   rss_matvec           : y = A x by FFT (the exact A of Eq. 3)
//   rss_solve_iterative  : PCG or right-preconditioned GMRES(m) with the RS-S
//                          factorization as preconditioner, to 1e-12 in the
//                          paper's experiments (Tables "laplace", "helmholtz").
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <mutex>
#include <vector>

#include "internal.h"

namespace {

constexpr int NTI = 256;

// ------------------------------------------------------------------ self-cell integral
// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n from the
// Chebyshev guesses cos(pi (i - 1/4) / (n + 1/2))).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

}  // namespace

rss_status self_integral(int kind, double h, double kappa, double* re, double* im) {
  if (!(h > 0)) {
    rss_set_error("rss_self_integral: h must be positive");
    return RSS_EINVAL;
  }
  const double a = 0.5 * h;
  if (kind == RSS_LAPLACE) {
    *re = -(1.0 / (2.0 * M_PI)) * 2.0 * a * a * (2.0 * std::log(a) + std::log(2.0) - 3.0 + 0.5 * M_PI);
    *im = 0.0;
    return RSS_OK;
  }
  if (kind == RSS_HELMHOLTZ || kind == RSS_HELMHOLTZ_LS) {
    if (!(kappa > 0)) {
      rss_set_error("rss_self_integral: kappa must be positive");
      return RSS_EINVAL;
    }
    // 8 (i/4) int_0^{pi/4} [rho H1(kappa rho)/kappa + 2i/(pi kappa^2)] dtheta, rho = a / cos(theta):
    // int_0^R rho H0(kappa rho) drho = R H1(kappa R)/kappa - lim_{rho->0} rho H1(kappa rho)/kappa,
    // and rho Y1(kappa rho) -> -2/(pi kappa).  The integrand is smooth on [0, pi/4].
    std::vector<double> gx, gw;
    gauss_legendre(48, gx, gw);
    double sr = 0.0, si = 0.0;
    for (int i = 0; i < 48; ++i) {
      const double t = 0.125 * M_PI * (gx[i] + 1.0), R = a / std::cos(t);
      sr += gw[i] * (R * ::j1(kappa * R) / kappa);
      si += gw[i] * (R * ::y1(kappa * R) / kappa + 2.0 / (M_PI * kappa * kappa));
    }
    sr *= 0.125 * M_PI;
    si *= 0.125 * M_PI;
    // (i/4) * 8 * (sr + i si) = 2 i sr - 2 si
    *re = -2.0 * si;
    *im = 2.0 * sr;
    return RSS_OK;
  }
  rss_set_error("rss_self_integral: kind must be RSS_LAPLACE, RSS_HELMHOLTZ or RSS_HELMHOLTZ_LS");
  return RSS_EINVAL;
}

extern "C" rss_status rss_self_integral(int kind, double h, double kappa, double* re, double* im) {
  if (!re || !im) {
    rss_set_error("rss_self_integral: NULL output");
    return RSS_EINVAL;
  }
  return self_integral(kind, h, kappa, re, im);
}

namespace {

// ------------------------------------------------------------------ FFT matvec
// On the s x s grid, (A x)_i = d_i x_i + w_i sum_{j != i} K(x_i - x_j) w_j x_j
// (w = 1 and d_i = A_ii except for Lippmann-Schwinger).  The sum is a 2D
// convolution with the kernel at displacements |dx|, |dy| <= s - 1, embedded in
// a 2s x 2s circulant and applied by FFT.
struct MatvecState {
  std::mutex mu;
  bool ready = false;
  int s = 0;
  cufftDoubleComplex* khat = nullptr;   // 2s x 2s spectrum of the circulant, divided by (2s)^2
  cufftHandle plan = 0;                 // 2D Z2Z, batch 1
  bool has_plan = false;
};

__global__ void k_circulant(cufftDoubleComplex* c, int s, KParams kp, Geo geo) {
  const long long m = 2LL * s, tot = m * m;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int cx = (int)(e % m), cy = (int)(e / m);
    const int dx = cx < s ? cx : cx - (int)m, dy = cy < s ? cy : cy - (int)m;   // wrap; |d| = s unused
    cufftDoubleComplex v{0.0, 0.0};
    if (!(dx == 0 && dy == 0) && dx != -s && dy != -s) {
      if (kp.kind == RSS_LAPLACE || kp.kind == RSS_TEST_RPOLY) {
        v.x = kval(kp, dx * geo.hg, dy * geo.hg, 0.0, 0.0, 0.0);
      } else {
        const zd z = kval(kp, dx * geo.hg, dy * geo.hg, 0.0, 0.0, zd{});
        v.x = z.x;
        v.y = z.y;
      }
    }
    c[e] = v;
  }
}

__global__ void k_scale_c(cufftDoubleComplex* c, long long n, double f) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    c[e].x *= f;
    c[e].y *= f;
  }
}

template <typename T> __device__ inline cufftDoubleComplex to_c(T v) {
  if constexpr (sizeof(T) == sizeof(double)) return cufftDoubleComplex{v, 0.0};
  else return cufftDoubleComplex{v.x, v.y};
}

// pad[g(i)] = w_i x_i on the zeroed 2s x 2s buffer
template <typename T>
__global__ void k_pad(const T* __restrict__ x, int64_t n, const int* __restrict__ u2g, int s,
                      const double* __restrict__ w, cufftDoubleComplex* __restrict__ pad) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int g = u2g[i], ix = g % s, iy = g / s;
    cufftDoubleComplex v = to_c(x[i]);
    if (w) {
      v.x *= w[g];
      v.y *= w[g];
    }
    pad[(size_t)iy * 2 * s + ix] = v;
  }
}

__global__ void k_mul_spec(cufftDoubleComplex* __restrict__ a, const cufftDoubleComplex* __restrict__ k, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const cufftDoubleComplex u = a[e], v = k[e];
    a[e] = cufftDoubleComplex{u.x * v.x - u.y * v.y, u.x * v.y + u.y * v.x};
  }
}

// y_i = w_i conv_i + d_i x_i
template <typename T>
__global__ void k_extract(const cufftDoubleComplex* __restrict__ pad, const T* __restrict__ x, T* __restrict__ y,
                          int64_t n, const int* __restrict__ u2g, int s, const double* __restrict__ w, KParams kp) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int g = u2g[i], ix = g % s, iy = g / s;
    cufftDoubleComplex v = pad[(size_t)iy * 2 * s + ix];
    if constexpr (sizeof(T) == sizeof(double)) {
      y[i] = v.x + kp.diag_re * x[i];
    } else {
      zd d{kp.diag_re, kp.diag_im};
      if (w) {
        const double wi = w[g];
        v.x *= wi;
        v.y *= wi;
        d = zd{1.0 + wi * wi * kp.diag_re, wi * wi * kp.diag_im};
      }
      y[i] = zd{v.x, v.y} + d * x[i];
    }
  }
}

rss_status matvec_state(const rss_factorization* fc, MatvecState** out, cudaStream_t st) {
  rss_factorization* f = const_cast<rss_factorization*>(fc);
  static std::mutex create_mu;
  {
    std::lock_guard<std::mutex> lk(create_mu);
    if (!f->mv) f->mv = new (std::nothrow) MatvecState();
  }
  MatvecState* m = static_cast<MatvecState*>(f->mv);
  if (!m) {
    rss_set_error("rss_matvec: host allocation failed");
    return RSS_ENOMEM;
  }
  std::lock_guard<std::mutex> lk(m->mu);
  if (!m->ready) {
    const int s = f->side;
    const size_t tot = (size_t)4 * s * s;
    RSS_CUDA(cudaMalloc(&m->khat, sizeof(cufftDoubleComplex) * tot));
    if (cufftPlan2d(&m->plan, 2 * s, 2 * s, CUFFT_Z2Z) != CUFFT_SUCCESS) {
      rss_set_error("rss_matvec: cuFFT plan creation failed");
      return RSS_ECUDA;
    }
    m->has_plan = true;
    KParams kp = f->kp;
    k_circulant<<<152 * 8, NTI, 0, st>>>(m->khat, s, kp, f->geo);
    RSS_LAUNCHED();
    if (cufftSetStream(m->plan, st) != CUFFT_SUCCESS || cufftExecZ2Z(m->plan, m->khat, m->khat, CUFFT_FORWARD) != CUFFT_SUCCESS) {
      rss_set_error("rss_matvec: cuFFT execution failed");
      return RSS_ECUDA;
    }
    k_scale_c<<<152 * 8, NTI, 0, st>>>(m->khat, (long long)tot, 1.0 / (double)tot);
    RSS_LAUNCHED();
    RSS_CUDA(cudaStreamSynchronize(st));
    m->s = s;
    m->ready = true;
  }
  *out = m;
  return RSS_OK;
}

template <typename T>
rss_status matvec_impl(const rss_factorization* f, const T* x, T* y, int64_t nrhs, int64_t ld, cudaStream_t st) {
  MatvecState* m = nullptr;
  rss_status s0 = matvec_state(f, &m, st);
  if (s0 != RSS_OK) return s0;
  const int s = m->s;
  const size_t tot = (size_t)4 * s * s;
  cufftDoubleComplex* pad = nullptr;
  RSS_CUDA(pool_malloc(reinterpret_cast<void**>(&pad), sizeof(cufftDoubleComplex) * tot, st));
  std::lock_guard<std::mutex> lk(m->mu);   // one plan: calls on the same factor are serialised
  rss_status res = RSS_OK;
  const unsigned g1 = std::min<long long>(cdiv(f->n, NTI), 152LL * 8), g2 = 152 * 8;
  for (int64_t q = 0; q < nrhs && res == RSS_OK; ++q) {
    if (cudaMemsetAsync(pad, 0, sizeof(cufftDoubleComplex) * tot, st) != cudaSuccess) { res = RSS_ECUDA; break; }
    k_pad<T><<<g1, NTI, 0, st>>>(x + q * ld, f->n, f->d_user_to_grid, s, f->d_w, pad);
    if (cufftSetStream(m->plan, st) != CUFFT_SUCCESS || cufftExecZ2Z(m->plan, pad, pad, CUFFT_FORWARD) != CUFFT_SUCCESS) {
      res = RSS_ECUDA;
      break;
    }
    k_mul_spec<<<g2, NTI, 0, st>>>(pad, m->khat, (long long)tot);
    if (cufftExecZ2Z(m->plan, pad, pad, CUFFT_INVERSE) != CUFFT_SUCCESS) { res = RSS_ECUDA; break; }
    k_extract<T><<<g1, NTI, 0, st>>>(pad, x + q * ld, y + q * ld, f->n, f->d_user_to_grid, s, f->d_w, f->kp);
    if (cudaGetLastError() != cudaSuccess) res = RSS_ECUDA;
  }
  pool_free(pad, st);
  if (res != RSS_OK) rss_set_error("rss_matvec: FFT or launch failure");
  return res;
}

// ------------------------------------------------------------------ vector kernels (deterministic reductions)
constexpr int RED_BLOCKS = 512;

template <typename T> __device__ inline double re_dot(T a, T b) {
  if constexpr (sizeof(T) == sizeof(double)) return a * b;
  else return a.x * b.x + a.y * b.y;
}
template <typename T> __device__ inline double im_dot(T a, T b) {
  if constexpr (sizeof(T) == sizeof(double)) return 0.0;
  else return a.x * b.y - a.y * b.x;
}

// partial sums of conj(a_i) b_i per block (fixed grid, fixed order)
template <typename T>
__global__ void __launch_bounds__(NTI) k_dot_part(const T* __restrict__ a, const T* __restrict__ b, int64_t n,
                                                  double2* __restrict__ part) {
  __shared__ double sr[NTI], si[NTI];
  double r = 0.0, im = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    r += re_dot(a[i], b[i]);
    im += im_dot(a[i], b[i]);
  }
  sr[threadIdx.x] = r;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int d = NTI / 2; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) {
      sr[threadIdx.x] += sr[threadIdx.x + d];
      si[threadIdx.x] += si[threadIdx.x + d];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = double2{sr[0], si[0]};
}

__global__ void k_dot_final(const double2* __restrict__ part, int np, double2* __restrict__ out) {
  __shared__ double sr[NTI], si[NTI];
  double r = 0.0, im = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    r += part[i].x;
    im += part[i].y;
  }
  sr[threadIdx.x] = r;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int d = NTI / 2; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) {
      sr[threadIdx.x] += sr[threadIdx.x + d];
      si[threadIdx.x] += si[threadIdx.x + d];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = double2{sr[0], si[0]};
}

// y = alpha x + beta y
template <typename T>
__global__ void k_axpby(T* __restrict__ y, const T* __restrict__ x, double ar, double ai, double br, double bi, int64_t n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if constexpr (sizeof(T) == sizeof(double)) {
      y[i] = ar * x[i] + br * y[i];
    } else {
      y[i] = zd{ar, ai} * x[i] + zd{br, bi} * y[i];
    }
  }
}

template <typename T> struct Vec {
  const rss_factorization* f;
  cudaStream_t st;
  double2* part;
  double2* res;
  int64_t n;
  unsigned grid() const { return std::min<long long>(cdiv(n, NTI), 152LL * 8); }
  // conj(a)^T b, synchronously
  rss_status dot(const T* a, const T* b, std::complex<double>* out) const {
    k_dot_part<T><<<RED_BLOCKS, NTI, 0, st>>>(a, b, n, part);
    k_dot_final<<<1, NTI, 0, st>>>(part, RED_BLOCKS, res);
    RSS_LAUNCHED();
    double2 h;
    RSS_CUDA(cudaMemcpyAsync(&h, res, sizeof(double2), cudaMemcpyDeviceToHost, st));
    RSS_CUDA(cudaStreamSynchronize(st));
    *out = std::complex<double>(h.x, h.y);
    return RSS_OK;
  }
  rss_status axpby(T* y, const T* x, std::complex<double> a, std::complex<double> b) const {
    k_axpby<T><<<grid(), NTI, 0, st>>>(y, x, a.real(), a.imag(), b.real(), b.imag(), n);
    RSS_LAUNCHED();
    return RSS_OK;
  }
  rss_status copy(T* y, const T* x) const {
    RSS_CUDA(cudaMemcpyAsync(y, x, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
    return RSS_OK;
  }
  rss_status A(const T* x, T* y) const { return matvec_impl<T>(f, x, y, 1, n, st); }
  rss_status Minv(const T* b, T* x) const {   // x = (factorization)^{-1} b
    RSS_CUDA(cudaMemcpyAsync(x, b, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
    return solve_impl<T>(f, x, 1, n, st);
  }
};

#define RSS_TRY(expr)                \
  do {                               \
    rss_status s_ = (expr);          \
    if (s_ != RSS_OK) return s_;     \
  } while (0)

// Preconditioned conjugate gradients (Hestenes-Stiefel) from x0 = M^{-1} b.
template <typename T>
rss_status pcg(const Vec<T>& v, const T* b, T* x, T* r, T* z, T* p, T* q, double tol, int maxit, int* iters,
               double* relres) {
  std::complex<double> t;
  RSS_TRY(v.dot(b, b, &t));
  const double nb = std::sqrt(t.real());
  RSS_TRY(v.Minv(b, x));
  RSS_TRY(v.A(x, q));
  RSS_TRY(v.copy(r, b));
  RSS_TRY(v.axpby(r, q, -1.0, 1.0));
  RSS_TRY(v.dot(r, r, &t));
  double rel = std::sqrt(t.real()) / nb;
  int it = 0;
  if (rel > tol) {
    RSS_TRY(v.Minv(r, z));
    RSS_TRY(v.copy(p, z));
    std::complex<double> rz;
    RSS_TRY(v.dot(r, z, &rz));
    while (it < maxit) {
      RSS_TRY(v.A(p, q));
      std::complex<double> pq;
      RSS_TRY(v.dot(p, q, &pq));
      const double alpha = rz.real() / pq.real();
      RSS_TRY(v.axpby(x, p, alpha, 1.0));
      RSS_TRY(v.axpby(r, q, -alpha, 1.0));
      ++it;
      RSS_TRY(v.dot(r, r, &t));
      rel = std::sqrt(t.real()) / nb;
      if (rel <= tol) break;
      RSS_TRY(v.Minv(r, z));
      std::complex<double> rz2;
      RSS_TRY(v.dot(r, z, &rz2));
      RSS_TRY(v.axpby(p, z, 1.0, rz2.real() / rz.real()));
      rz = rz2;
    }
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;
  return RSS_OK;
}

// Right-preconditioned GMRES(m) from x0 = M^{-1} b: A M^{-1} u = b, x = M^{-1} u;
// Arnoldi with modified Gram-Schmidt, Givens rotations on the Hessenberg matrix.
template <typename T>
rss_status gmres(const Vec<T>& v, const T* b, T* x, T* r, T* w, T* tmp, T* V, int m, double tol, int maxit,
                 int* iters, double* relres) {
  using C = std::complex<double>;
  const int64_t n = v.n;
  C t;
  RSS_TRY(v.dot(b, b, &t));
  const double nb = std::sqrt(t.real());
  RSS_TRY(v.Minv(b, x));
  int it = 0;
  double rel = 0.0;
  std::vector<C> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  while (true) {
    RSS_TRY(v.A(x, w));
    RSS_TRY(v.copy(r, b));
    RSS_TRY(v.axpby(r, w, -1.0, 1.0));
    RSS_TRY(v.dot(r, r, &t));
    const double beta = std::sqrt(t.real());
    rel = beta / nb;
    if (rel <= tol || it >= maxit || beta == 0.0) break;
    RSS_TRY(v.axpby(V, r, 1.0 / beta, 0.0));
    std::fill(g.begin(), g.end(), C(0.0));
    g[0] = beta;
    int jd = 0;
    for (int j = 0; j < m; ++j) {
      T* vj = V + (size_t)j * n;
      RSS_TRY(v.Minv(vj, tmp));
      RSS_TRY(v.A(tmp, w));
      for (int i = 0; i <= j; ++i) {
        C h;
        RSS_TRY(v.dot(V + (size_t)i * n, w, &h));
        H[(size_t)i * m + j] = h;
        RSS_TRY(v.axpby(w, V + (size_t)i * n, -h, 1.0));
      }
      RSS_TRY(v.dot(w, w, &t));
      const double hn = std::sqrt(t.real());
      H[(size_t)(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        const C a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + j] = -std::conj(sn[i]) * a + std::conj(cs[i]) * c;
      }
      const C hjj = H[(size_t)j * m + j], hj1 = H[(size_t)(j + 1) * m + j];
      const double den = std::sqrt(std::norm(hjj) + std::norm(hj1));
      cs[j] = den > 0 ? hjj / den : C(1.0);
      sn[j] = den > 0 ? hj1 / den : C(0.0);
      H[(size_t)j * m + j] = std::conj(cs[j]) * hjj + std::conj(sn[j]) * hj1;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -std::conj(sn[j]) * g[j];
      g[j] = std::conj(cs[j]) * g[j];
      ++it;
      jd = j + 1;
      if (std::abs(g[j + 1]) / nb <= tol || it >= maxit || hn == 0.0) break;
      RSS_TRY(v.axpby(V + (size_t)(j + 1) * n, w, 1.0 / hn, 0.0));
    }
    for (int i = jd - 1; i >= 0; --i) {   // back substitution on the triangular H
      C s = g[i];
      for (int l = i + 1; l < jd; ++l) s -= H[(size_t)i * m + l] * y[l];
      y[i] = s / H[(size_t)i * m + i];
    }
    // u = V y; x += M^{-1} u
    RSS_TRY(v.axpby(w, V, y[0], 0.0));
    for (int i = 1; i < jd; ++i) RSS_TRY(v.axpby(w, V + (size_t)i * n, y[i], 1.0));
    RSS_TRY(v.Minv(w, tmp));
    RSS_TRY(v.axpby(x, tmp, 1.0, 1.0));
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;
  return RSS_OK;
}

template <typename T>
rss_status iterative_impl(const rss_factorization* f, const T* b, T* x, double tol, int maxit, int restart, int method,
                          int* iters, double* relres, cudaStream_t st) {
  const int64_t n = f->n;
  const int m = restart > 0 ? restart : 20;
  const bool use_cg = method == 1 || (method == 0 && sizeof(T) == sizeof(double));
  const size_t nvec = use_cg ? 4 : 3 + (size_t)m + 1;
  char* mem = nullptr;
  const size_t vb = (sizeof(T) * (size_t)n + 255) & ~size_t(255);
  RSS_CUDA(pool_malloc(reinterpret_cast<void**>(&mem), vb * nvec + sizeof(double2) * (RED_BLOCKS + 1), st));
  T* w0 = reinterpret_cast<T*>(mem);
  auto vec = [&](size_t i) { return reinterpret_cast<T*>(mem + i * vb); };
  Vec<T> v{f, st, reinterpret_cast<double2*>(mem + vb * nvec), reinterpret_cast<double2*>(mem + vb * nvec) + RED_BLOCKS, n};
  rss_status s = use_cg ? pcg<T>(v, b, x, w0, vec(1), vec(2), vec(3), tol, maxit, iters, relres)
                        : gmres<T>(v, b, x, w0, vec(1), vec(2), vec(3), m, tol, maxit, iters, relres);
  pool_free(mem, st);
  cudaStreamSynchronize(st);
  return s;
}

bool device_ptr(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

}  // namespace

void free_matvec(rss_factorization* f) {
  MatvecState* m = static_cast<MatvecState*>(f->mv);
  if (!m) return;
  if (m->has_plan) cufftDestroy(m->plan);
  if (m->khat) cudaFree(m->khat);
  delete m;
  f->mv = nullptr;
}

extern "C" rss_status rss_matvec(const rss_factorization* f, const void* x, void* y, int64_t nrhs, int64_t ld,
                                 void* stream) {
  if (!f || f->tag != RSS_TAG_FACTOR) {
    rss_set_error("rss_matvec: not a factor handle");
    return RSS_EINVAL;
  }
  if (!x || !y || nrhs <= 0 || ld < f->n) {
    rss_set_error("rss_matvec: x and y must be non-NULL with nrhs > 0 and ld >= n");
    return RSS_EINVAL;
  }
  if (f->kp.kind == RSS_TEST_POLY) {
    rss_set_error("rss_matvec: the phase-weighted test kernel is not a convolution");
    return RSS_EINVAL;
  }
  if (!device_ptr(x) || !device_ptr(y)) {
    rss_set_error("rss_matvec: x and y must be device memory");
    return RSS_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return f->is_complex ? matvec_impl<zd>(f, static_cast<const zd*>(x), static_cast<zd*>(y), nrhs, ld, st)
                       : matvec_impl<double>(f, static_cast<const double*>(x), static_cast<double*>(y), nrhs, ld, st);
}

extern "C" rss_status rss_solve_iterative(const rss_factorization* f, const void* b, void* x, double tol, int maxit,
                                          int restart, int method, int* iters, double* relres, void* stream) {
  if (!f || f->tag != RSS_TAG_FACTOR) {
    rss_set_error("rss_solve_iterative: not a factor handle");
    return RSS_EINVAL;
  }
  if (!b || !x || b == x || !(tol > 0) || method < 0 || method > 2 || restart > 1000) {
    rss_set_error("rss_solve_iterative: b and x must be distinct non-NULL buffers, tol > 0, method 0..2");
    return RSS_EINVAL;
  }
  if (f->kp.kind == RSS_TEST_POLY) {
    rss_set_error("rss_solve_iterative: the phase-weighted test kernel has no FFT matvec");
    return RSS_EINVAL;
  }
  if (!device_ptr(b) || !device_ptr(x)) {
    rss_set_error("rss_solve_iterative: b and x must be device memory");
    return RSS_EINVAL;
  }
  const int mi = maxit > 0 ? maxit : 200;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return f->is_complex ? iterative_impl<zd>(f, static_cast<const zd*>(b), static_cast<zd*>(x), tol, mi, restart,
                                            method, iters, relres, st)
                       : iterative_impl<double>(f, static_cast<const double*>(b), static_cast<double*>(x), tol, mi,
                                                restart, method, iters, relres, st);
}
