// RS-S factorization on the device (Algorithm 1), batched by colour class.
//
// Per level (box grid side g >= 4) and per colour class (ix mod 3, iy mod 3),
// all boxes of the class are pairwise more than distance 2 apart (Section 3),
// so each phase handles the whole class in one launch:
//   k_id      : proxy stack Y = [A_MB; K_PB; A_BM^*; K_BP^*] (Eqs. 4-6) and its
//               column-pivoted Householder QR, truncated at eps (Definition 1);
//   k_elim    : sparsification (Eq. 7), LU of X_RR, E = X_CR U^{-1} and
//               F = L^{-1} P X_RC (Eq. 8);
//   k_schur   : A_CC -= E F scattered into the stencil blocks (Remark 2);
// then the merge to the parent level (Section 2.4) and a dense LU at the top.
//
// Matrix storage: for each box u of a level, 25 blocks A(u, v), v = u + (dx, dy),
// |dx|, |dy| <= 2, each nmax x nmax column-major over the level-start point
// lists of u and v.  A box's active points are a position list into its
// level-start list (the skeleton after elimination); far pairs (distance > 2)
// are never stored because they are never modified (Theorem 1).
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <type_traits>
#include <vector>

#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "internal.h"
#include "tc_gemm.cuh"

namespace {

// Pivot ties: remaining squared norms within TIE_REL n_max + TIE_ABS sqrt(n_max y2max)
// of the maximum n_max (y2max: largest initial squared column norm) are rounding
// noise apart and count as tied; the lowest original column wins.
constexpr double TIE_REL = 1e-6;
constexpr double TIE_ABS = 1e-12;
// A downdated squared norm is re-accumulated once it falls below sqrt(unit
// roundoff) of its last accumulated value (LAPACK geqp3's rule); between
// re-accumulations it is accurate to a few 1e-8 relative, inside the tie window.
constexpr double RECOMPUTE_REL = 1.4901161193847656e-08;
constexpr int NT = 256;                 // threads per CTA for the per-box kernels

template <typename T> struct LevelDev {
  int g, nbox, nmax;
  int* pts;    // nbox x nmax tree indices (level-start points)
  int* n;      // nbox
  int* act;    // nbox x nmax active positions
  int* nact;   // nbox
  T* blk;      // nbox x 25 x nmax x nmax
};

__device__ __forceinline__ int nbr_box(int u, int g, int dx, int dy) {
  int bx = u % g + dx, by = u / g + dy;
  return (bx < 0 || by < 0 || bx >= g || by >= g) ? -1 : by * g + bx;
}
__device__ __forceinline__ int off_index(int u, int v, int g) {
  return (v / g - u / g + 2) * 5 + (v % g - u % g + 2);
}
__device__ __forceinline__ int cheb(int u, int v, int g) {
  return max(abs(u % g - v % g), abs(u / g - v / g));
}

template <typename T> __device__ T block_sum(T v, T* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? sh[lane] : zero<T>();
    v = warp_sum(v);
    if (lane == 0) sh[0] = v;
  }
  __syncthreads();
  return sh[0];
}

__device__ inline double warp_max(double v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, d));
  return v;
}

// ------------------------------------------------------------------ kernel table
// tab[(dy + s - 1) (2s - 1) + (dx + s - 1)] = K at grid displacement (dx, dy) != 0.
template <typename T> __global__ void k_ktab(T* tab, int side, KParams kp, Geo geo) {
  const long long w = 2 * side - 1, tot = w * w;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int dx = (int)(e % w) - (side - 1), dy = (int)(e / w) - (side - 1);
    tab[e] = (dx == 0 && dy == 0) ? zero<T>() : kval(kp, dx * geo.hg, dy * geo.hg, 0.0, 0.0, T{});
  }
}

// Lippmann-Schwinger weights w = kappa sqrt(b(x)) = kappa exp(-bump_a |x - c|^2 / 2)
// at each grid point (iy * side + ix)   (Eq. 19)
__global__ void k_ls_weights(double* w, int side, Geo geo, double kappa, double cx, double cy, double a) {
  const long long n = (long long)side * side;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double x = geo.x0 + (e % side) * geo.hg - cx, y = geo.y0 + (e / side) * geo.hg - cy;
    w[e] = kappa * exp(-0.5 * a * (x * x + y * y));
  }
}

// ------------------------------------------------------------------ leaf generation
template <typename T>
__global__ void __launch_bounds__(NT) k_gen_blocks(LevelDev<T> L, const int2* __restrict__ ixy,
                                                   const T* __restrict__ tab, KParams kp, int side) {
  const int u = blockIdx.x / 25, o = blockIdx.x % 25;
  const int v = nbr_box(u, L.g, o % 5 - 2, o / 5 - 2);
  if (v < 0) return;
  const int nu = L.n[u], nv = L.n[v];
  // grid coordinates of both boxes' points, read once (leaf boxes: at most 256 points)
  __shared__ int2 gu[256], gv[256];
  for (int i = threadIdx.x; i < nu; i += blockDim.x) gu[i] = ixy[L.pts[u * L.nmax + i]];
  for (int j = threadIdx.x; j < nv; j += blockDim.x) gv[j] = ixy[L.pts[v * L.nmax + j]];
  __syncthreads();
  T* A = L.blk + ((size_t)u * 25 + o) * L.nmax * L.nmax;
  if (nu == 0) return;
  // entry e = i + j nu, stepped by the block size without a division per entry
  const int di = (int)blockDim.x % nu, dj = (int)blockDim.x / nu;
  int i = (int)threadIdx.x % nu, j = (int)threadIdx.x / nu;
  for (; j < nv; i += di, j += dj) {
    if (i >= nu) {
      i -= nu;
      ++j;
      if (j >= nv) break;
    }
    A[(size_t)j * L.nmax + i] = aval_tab<T>(kp, tab, side, gu[i], gv[j]);
  }
}

// ------------------------------------------------------------------ ID (Definition 1, Eq. 6)
// One CTA per box.  Y = [A_MB; K_PB; A_BM^*; K_BP^*] is assembled once and then
// only read: the Householder reflectors H_l = I - tau_l v_l v_l^H are kept as
// V (m x k) and G (n x k) with H_{j-1}..H_0 Y = Y - V G^T (column c of G holds
// tau_l v_l^H (H_{l-1}..H_0 Y)[:, c]), so a step costs one product v^H Y over
// the remaining columns plus O((m + n) j) corrections, the pivot column and row j
// of R are formed on demand, and Y is never rewritten.  In exact arithmetic this
// is the same sequence of reflectors and pivots as updating Y in place.
constexpr int NT_ID = 256;
// Cluster ID (small colour classes): up to CL_QMAX CTAs per box (above 8 a
// non-portable cluster size), NTC threads per CTA: 512 when every CTA of the
// launch gets an SM of its own (more warps share the per-step dot products of
// the reflector with the owned rows), else 256, two CTAs per SM.
constexpr int CL_QMAX = 16;
constexpr int CL_QDEF = 8;   // the largest size the default policy takes
// stride of one of the two partial-sum buffers of the cluster ID: a vector of up
// to 2 nmax sums, or 2 scalars plus one partial per warp
template <int NTC> __host__ __device__ inline int cl_part_stride(int nmax) {
  return 2 * nmax > 2 + NTC / 32 ? 2 * nmax : 2 + NTC / 32;
}

// T: arithmetic of the ID; S: scalar of the matrix.  T = double with S = zd is
// the complex symmetric case (Helmholtz): there A_BM^* = conj(A_MB) and
// K_BP^* = conj(K_PB) hold through the eliminations (T stays real, so the
// Schur updates keep A complex symmetric), the stack is [X; conj X] with
// X = [A_MB; K_PB], and its Gram matrix 2 Re(X^H X) is that of the real matrix
// sqrt(2) [Re X; Im X].  Column-pivoted QR sees Y only through its Gram matrix
// (norms, pivots, R up to unimodular row scales, ||R22||, T = R11^{-1} R12), so
// the real stack [Re X; Im X] gives the same ID with T real, at a quarter of
// the arithmetic.
template <typename T, typename S = T> struct IdArgs {
  LevelDev<S> L;
  const int* boxes;   // colour class
  int base;           // first box of this chunk within the class
  T* ws;              // chunk workspace: per box Y (ldY x nmax), V (ldY x nmax), G, Rr (nmax x nmax)
  int ldY;
  int half;           // 1: rows [A_MB; K_PB] only (real symmetric kernel)
  int* k_out;         // per class box
  int* perm_out;      // class x nmax
  S* T_ws;            // class x nmax x nmax (k x r, ld nmax)
  const int2* ixy;
  KParams kp;
  Geo geo;
  double eps;
  int P;              // proxy points
  double rho;         // proxy radius
  double Lbox;        // box side
  int g_sm;           // 1: G (nmax x nmax) and row k of V are kept in shared memory
  const S* ptab;      // proxy rows K(y_p, x) by the point's place in its box (null: evaluated here)
  int lsz;            // grid points per box side at this level
};

template <typename T, typename S> __device__ inline S id_store(T v) {
  if constexpr (std::is_same<T, S>::value) return v;
  else return S{v, 0.0};
}
template <typename T, typename S> __device__ inline T id_load(S v) {
  if constexpr (std::is_same<T, S>::value) return v;
  else return v.x;
}

// Entry (i, j) of the proxy stack of box B (Eq. 6): rows [A_MB; K_PB] then
// [A_BM^*; K_BP^*]; with T real and S complex, [Re X; Im X] for X = [A_MB; K_PB].
// Mbox/Moff: the distance-2 boxes and their row offsets, mh = their active rows,
// (cx, cy) the box centre; column j is point j of B (identity active list).
template <typename T, typename S>
__device__ __forceinline__ T id_entry(const IdArgs<T, S>& a, int B, int i, int j, int mh, const int* Mbox,
                                      const int* Moff, double cx, double cy) {
  const LevelDev<S>& L = a.L;
  const int nmax = L.nmax, g = L.g, P = a.P;
  const size_t nn = (size_t)nmax * nmax;
  constexpr bool split = !std::is_same<T, S>::value;
  bool second = i >= mh + P;                // conjugate half (or imaginary parts)
  const int ii = second ? i - mh - P : i;   // row of X
  S v;
  if (ii < mh) {
    int q = 0;
    while (Moff[q + 1] <= ii) ++q;
    const int mb = Mbox[q];
    const int pm = L.act[mb * nmax + (ii - Moff[q])];
    if (split || !second)
      v = L.blk[((size_t)mb * 25 + off_index(mb, B, g)) * nn + (size_t)j * nmax + pm];
    else
      v = cj(L.blk[((size_t)B * 25 + off_index(B, mb, g)) * nn + (size_t)pm * nmax + j]);
  } else {
    const int p = ii - mh;
    const int2 q = a.ixy[L.pts[B * nmax + j]];
    if (a.ptab != nullptr && (split || !second)) {   // K(y_p, x_j) from the level's table
      const int local = (q.y - (B / g) * a.lsz) * a.lsz + (q.x - (B % g) * a.lsz);
      v = a.ptab[(size_t)p * a.lsz * a.lsz + local];
    } else {
      double sn, cs;
      sincospi(2.0 * p / P, &sn, &cs);
      const double px = cx + a.rho * cs, py = cy + a.rho * sn;
      const double xj = a.geo.x0 + q.x * a.geo.hg, yj = a.geo.y0 + q.y * a.geo.hg;
      v = (!split && second) ? cj(kval(a.kp, xj, yj, px, py, S{})) : kval(a.kp, px, py, xj, yj, S{});
    }
    if (a.kp.kind == RSS_HELMHOLTZ_LS)   // proxy weight kappa, column weight w_j
      v = (a.kp.kappa * a.kp.w[q.y * a.geo.side + q.x]) * v;
  }
  if constexpr (split) return second ? v.y : v.x;
  else return v;
}

// Proxy rows by place (Eq. 6): on the uniform grid the box centre, the proxy
// circle and the box's grid points move together from box to box, and every
// kernel kind depends only on x - y, so K(y_p, x) for a point x of box B is a
// function of p and of x's place (ox, oy) inside B (lsz x lsz places): one table
// per level, tab[p * lsz^2 + oy * lsz + ox], serves the proxy rows of every box.
// The coordinates are taken relative to the box centre, y_p - x =
// rho (cos, sin)(2 pi p / P) - ((ox, oy) + 1/2 - lsz/2) hg.
template <typename S>
__global__ void __launch_bounds__(NT) k_proxy_tab(S* __restrict__ tab, int lsz, int P, double rho, double hg,
                                                  KParams kp) {
  const long long nloc = (long long)lsz * lsz, tot = nloc * P;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(e / nloc), o = (int)(e % nloc), ox = o % lsz, oy = o / lsz;
    double sn, cs;
    sincospi(2.0 * p / P, &sn, &cs);
    const double xr = (ox + 0.5 - 0.5 * lsz) * hg, yr = (oy + 0.5 - 0.5 * lsz) * hg;
    tab[e] = kval(kp, rho * cs - xr, rho * sn - yr, 0.0, 0.0, S{});
  }
}

template <typename T, typename S = T> __global__ void __launch_bounds__(NT_ID, 4) k_id(IdArgs<T, S> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const LevelDev<S>& L = a.L;
  const int nmax = L.nmax, g = L.g, ldY = a.ldY;
  T* vbuf = reinterpret_cast<T*>(smraw);          // ldY: current reflector
  T* u = vbuf + ldY;                              // nmax: V^H v
  T* beta = u + nmax;                             // nmax: R diagonal
  double* norms2 = reinterpret_cast<double*>(beta + nmax);
  double* ref = norms2 + nmax;
  double* taus = ref + nmax;
  int* perm = reinterpret_cast<int*>(taus + nmax);
  int* flag = perm + nmax;
  T* Gs = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(smraw) +
                               ((reinterpret_cast<unsigned char*>(flag + nmax) - smraw + 15) & ~size_t(15)));
  T* vrow = Gs + (size_t)nmax * nmax;             // row k of V (a.g_sm)
  __shared__ int Mbox[16], Moff[17], s_nM, s_piv, s_stop;
  __shared__ double s_thresh, s_y2max, s_redd[32];
  __shared__ T s_scale;

  const int bi = a.base + blockIdx.x;
  const int B = a.boxes[bi];
  const size_t nn = (size_t)nmax * nmax;
  const int n = L.n[B];
  const size_t slot = 2 * (size_t)ldY * nmax + 2 * nn;
  const T* Y = a.ws + (size_t)blockIdx.x * slot;
  T* Yw = a.ws + (size_t)blockIdx.x * slot;
  T* V = Yw + (size_t)ldY * nmax;
  T* G = a.g_sm ? Gs : V + (size_t)ldY * nmax;   // G[l * nmax + c]
  T* Rr = V + (size_t)ldY * nmax + nn;            // Rr[i * nmax + c]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;

  if (tid == 0) {
    int cnt = 0, off = 0;
    for (int dy = -2; dy <= 2; ++dy)
      for (int dx = -2; dx <= 2; ++dx) {
        if (max(abs(dx), abs(dy)) != 2) continue;
        const int mb = nbr_box(B, g, dx, dy);
        if (mb < 0) continue;
        Mbox[cnt] = mb;
        Moff[cnt] = off;
        off += L.nact[mb];
        ++cnt;
      }
    Moff[cnt] = off;
    s_nM = cnt;
  }
  __syncthreads();
  const int nM = s_nM, mh = Moff[nM], P = a.P;
  const int m = a.half ? mh + P : 2 * (mh + P);
  const int bx = B % g, by = B / g;
  const double cx = a.geo.x0 - 0.5 * a.geo.hg + (bx + 0.5) * a.Lbox;
  const double cy = a.geo.y0 - 0.5 * a.geo.hg + (by + 0.5) * a.Lbox;

  // Y, column-major; column j = point j of B (not yet eliminated: identity active list)
  for (long long e = tid; e < (long long)m * n; e += blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    Yw[(size_t)j * ldY + i] = id_entry(a, B, i, j, mh, Mbox, Moff, cx, cy);
  }
  __syncthreads();
  for (int c = warp; c < n; c += nwarp) {
    double s = 0.0;
    for (int i = lane; i < m; i += 32) s += abs2(Y[(size_t)c * ldY + i]);
    s = warp_sum(s);
    if (lane == 0) {
      norms2[c] = s;
      ref[c] = s;
      perm[c] = c;
    }
  }
  __syncthreads();
  if (warp == 0) {
    double s = 0.0, mx = 0.0;
    for (int c = lane; c < n; c += 32) {
      s += norms2[c];
      mx = fmax(mx, norms2[c]);
    }
    s = warp_sum(s);
    mx = warp_max(mx);
    if (lane == 0) {
      s_thresh = a.eps * a.eps * s;
      s_y2max = mx;
    }
  }
  __syncthreads();

  int k = 0;
  const int kmax = min(m, n);
  while (k < kmax) {
    // stop test and pivot: largest remaining norm, lowest original column among ties
    if (warp == 0) {
      double s = 0.0, mx = -1.0;
      for (int c = k + lane; c < n; c += 32) {
        s += norms2[c];
        mx = fmax(mx, norms2[c]);
      }
      s = warp_sum(s);
      mx = warp_max(mx);
      const double thr = mx - (TIE_REL * mx + TIE_ABS * sqrt(mx * s_y2max));
      int bp = INT_MAX, bc = -1;
      for (int c = k + lane; c < n; c += 32)
        if (norms2[c] >= thr && perm[c] < bp) {
          bp = perm[c];
          bc = c;
        }
      for (int d = 16; d > 0; d >>= 1) {
        const int op = __shfl_xor_sync(0xffffffffu, bp, d), oc = __shfl_xor_sync(0xffffffffu, bc, d);
        if (op < bp) {
          bp = op;
          bc = oc;
        }
      }
      if (lane == 0) {
        s_stop = (s <= s_thresh) || bc < 0;   // bc < 0 only if every norm is NaN
        s_piv = bc;
        if (!s_stop && bc != k) {
          int ti = perm[k]; perm[k] = perm[bc]; perm[bc] = ti;
          double td = norms2[k]; norms2[k] = norms2[bc]; norms2[bc] = td;
          td = ref[k]; ref[k] = ref[bc]; ref[bc] = td;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int q = perm[k];
    // pivot column after k reflectors, rows k..m-1
    double s2 = 0.0;
    for (int i = k + tid; i < m; i += blockDim.x) {
      T x = Y[(size_t)q * ldY + i];
      for (int l = 0; l < k; ++l) x = msb(x, V[(size_t)l * ldY + i], G[(size_t)l * nmax + q]);
      vbuf[i] = x;
      s2 += abs2(x);
    }
    const double alpha2 = block_sum(s2, s_redd);
    if (tid == 0) {
      const T x0 = vbuf[k];
      const double alpha = sqrt(alpha2);
      if (alpha == 0.0) {
        s_stop = 1;
      } else {
        const double ax0 = sqrt(abs2(x0));
        T phase = from_re<T>(1.0);
        if (ax0 != 0.0) phase = scl(1.0 / ax0, x0);
        const T bt = scl(-alpha, phase);
        beta[k] = bt;
        s_scale = dv(from_re<T>(1.0), x0 - bt);   // 1 / (x0 - beta), one division
        taus[k] = (alpha + ax0) / alpha;
      }
    }
    __syncthreads();
    if (s_stop) break;
    {
      const T d = s_scale;
      for (int i = k + 1 + tid; i < m; i += blockDim.x) {
        const T v = vbuf[i] * d;
        vbuf[i] = v;
        V[(size_t)k * ldY + i] = v;
      }
      if (tid == 0) {
        vbuf[k] = from_re<T>(1.0);
        V[(size_t)k * ldY + k] = from_re<T>(1.0);
      }
    }
    __syncthreads();
    // u_l = v^H V[:, l] (l < k) and raw g_c = v^H Y[:, c] for the remaining columns,
    // four columns per warp: one accumulator per column and lane, then a transposing
    // butterfly that sums the four columns with six additions instead of twenty
    // (an FP64 instruction costs the same with one lane or 32)
    const int nc = n - k - 1, ncol = k + nc;
    for (int gi = warp; 4 * gi < ncol; gi += nwarp) {
      const T* col[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int w = 4 * gi + c;
        col[c] = w >= ncol ? nullptr : w < k ? V + (size_t)w * ldY : Y + (size_t)perm[k + 1 + (w - k)] * ldY;
      }
      T d[4] = {zero<T>(), zero<T>(), zero<T>(), zero<T>()};
      if (col[3] != nullptr) {
        for (int i = k + lane; i < m; i += 32) {
          const T x = vbuf[i];
#pragma unroll
          for (int c = 0; c < 4; ++c) d[c] = madc(d[c], x, col[c][i]);
        }
      } else {
        for (int i = k + lane; i < m; i += 32) {
          const T x = vbuf[i];
#pragma unroll
          for (int c = 0; c < 3; ++c)
            if (col[c] != nullptr) d[c] = madc(d[c], x, col[c][i]);
        }
      }
      // lanes 0-15 keep columns 0, 1 and lanes 16-31 columns 2, 3; then each group of
      // eight lanes keeps one column (lanes 8c .. 8c + 7: column c) and sums it
      const bool hi = lane >= 16;
      T a0 = hi ? d[2] : d[0], a1 = hi ? d[3] : d[1];
      a0 = a0 + shfl_xor(hi ? d[0] : d[2], 16);
      a1 = a1 + shfl_xor(hi ? d[1] : d[3], 16);
      const bool odd = (lane & 8) != 0;
      T t = odd ? a1 : a0;
      t = t + shfl_xor(odd ? a0 : a1, 8);
      t = t + shfl_xor(t, 4);
      t = t + shfl_xor(t, 2);
      t = t + shfl_xor(t, 1);
      const int w = 4 * gi + (lane >> 3);
      if ((lane & 7) == 0 && w < ncol) {
        if (w < k) u[w] = t;
        else G[(size_t)k * nmax + perm[k + 1 + (w - k)]] = t;
      }
    }
    if (a.g_sm)
      for (int l = tid; l <= k; l += blockDim.x) vrow[l] = V[(size_t)l * ldY + k];
    __syncthreads();
    // g_c, row k of R, norm downdate
    const double tau = taus[k];
    for (int pos = k + 1 + tid; pos < n; pos += blockDim.x) {
      const int c = perm[pos];
      T gc = G[(size_t)k * nmax + c];
      for (int l = 0; l < k; ++l) gc = msb(gc, G[(size_t)l * nmax + c], u[l]);
      gc = scl(tau, gc);
      G[(size_t)k * nmax + c] = gc;
      T r = Y[(size_t)c * ldY + k];
      if (a.g_sm)
        for (int l = 0; l <= k; ++l) r = msb(r, vrow[l], G[(size_t)l * nmax + c]);
      else
        for (int l = 0; l <= k; ++l) r = msb(r, V[(size_t)l * ldY + k], G[(size_t)l * nmax + c]);
      Rr[(size_t)k * nmax + c] = r;
      const double nv = norms2[pos] - abs2(r);
      flag[pos] = nv < RECOMPUTE_REL * ref[pos];
      norms2[pos] = nv;
    }
    __syncthreads();
    for (int pos = k + 1 + warp; pos < n; pos += nwarp) {
      if (!flag[pos]) continue;
      const int c = perm[pos];
      double t = 0.0;
      int i = k + 1 + lane;
      for (; i + 96 < m; i += 128) {   // four rows per lane in flight
        T x0 = Y[(size_t)c * ldY + i], x1 = Y[(size_t)c * ldY + i + 32];
        T x2 = Y[(size_t)c * ldY + i + 64], x3 = Y[(size_t)c * ldY + i + 96];
        for (int l = 0; l <= k; ++l) {
          const T gl = G[(size_t)l * nmax + c];
          const T* vl = V + (size_t)l * ldY + i;
          x0 = msb(x0, vl[0], gl);
          x1 = msb(x1, vl[32], gl);
          x2 = msb(x2, vl[64], gl);
          x3 = msb(x3, vl[96], gl);
        }
        t += (abs2(x0) + abs2(x1)) + (abs2(x2) + abs2(x3));
      }
      for (; i < m; i += 32) {
        T x = Y[(size_t)c * ldY + i];
        for (int l = 0; l <= k; ++l) x = msb(x, V[(size_t)l * ldY + i], G[(size_t)l * nmax + c]);
        t += abs2(x);
      }
      t = warp_sum(t);
      if (lane == 0) {
        norms2[pos] = t;
        ref[pos] = t;
      }
    }
    __syncthreads();
    ++k;
  }
  __syncthreads();
  // T = R11^{-1} R12 (back substitution), k x r with ld nmax
  const int r = n - k;
  S* Tw = a.T_ws + (size_t)bi * nn;
  for (int c = tid; c < r; c += blockDim.x) {
    const int oc = perm[k + c];
    for (int i = k - 1; i >= 0; --i) {
      T x = Rr[(size_t)i * nmax + oc];
      for (int l = i + 1; l < k; ++l)
        x = msb(x, Rr[(size_t)i * nmax + perm[l]], id_load<T, S>(Tw[(size_t)c * nmax + l]));
      Tw[(size_t)c * nmax + i] = id_store<T, S>(dv(x, beta[i]));
    }
  }
  for (int c = tid; c < n; c += blockDim.x) a.perm_out[(size_t)bi * nmax + c] = perm[c];
  if (tid == 0) a.k_out[bi] = k;
}

// ------------------------------------------------------------------ ID on a thread-block cluster
// For colour classes too small to fill the GPU: a cluster of Q CTAs works on one
// box, CTA q owning a contiguous slice of the rows of Y (and of V).  Every CTA
// keeps an identical copy of the small state (norms, permutation, G, rows of R)
// and makes the same decisions; the sums over rows (column norms, the pivot
// column's norm, v^H Y, v^H V, re-accumulated norms) are formed per CTA and
// added through distributed shared memory in rank order, so all CTAs see the
// same bits.  Every CTA reaches every cluster barrier the same number of times.
template <typename T, typename S, int NTC>
__global__ void __launch_bounds__(NTC, (sizeof(T) == sizeof(double) && NTC == 256) ? 2 : 1) k_id_cl(IdArgs<T, S> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int Q = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const LevelDev<S>& L = a.L;
  const int nmax = L.nmax, g = L.g, ldY = a.ldY;
  const int rp = (ldY + Q - 1) / Q;                // rows per CTA (upper bound)
  T* vbuf = reinterpret_cast<T*>(smraw);           // rp: owned rows of the reflector
  T* u = vbuf + rp;                                // nmax
  T* beta = u + nmax;                              // nmax
  const int pst = cl_part_stride<NTC>(nmax);
  T* part = beta + nmax;                           // 2 x pst: partial sums, double buffered
  double* norms2 = reinterpret_cast<double*>(part + 2 * pst);
  double* ref = norms2 + nmax;
  double* taus = ref + nmax;
  int* perm = reinterpret_cast<int*>(taus + nmax);
  int* flag = perm + nmax;
  T* Gs = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(smraw) +
                               ((reinterpret_cast<unsigned char*>(flag + nmax) - smraw + 15) & ~size_t(15)));
  T* vrow = Gs + (size_t)nmax * nmax;              // row k of V (a.g_sm)
  __shared__ int Mbox[16], Moff[17], s_nM, s_stop;
  __shared__ double s_thresh, s_y2max;
  __shared__ T s_scale;

  const int box_local = blockIdx.x / Q;
  const int bi = a.base + box_local;
  const int B = a.boxes[bi];
  const size_t nn = (size_t)nmax * nmax;
  const int n = L.n[B];
  const size_t slot = 2 * (size_t)ldY * nmax + 2 * nn * Q;
  T* Yw = a.ws + (size_t)box_local * slot;
  const T* Y = Yw;
  T* V = Yw + (size_t)ldY * nmax;
  T* G = a.g_sm ? Gs : V + (size_t)ldY * nmax + 2 * nn * rank;   // this CTA's copy: G[l * nmax + c]
  T* Rr = V + (size_t)ldY * nmax + 2 * nn * rank + nn;            // Rr[i * nmax + c]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  int pb = 0;                                       // partial-sum buffer in use

  // sum the Q CTAs' partial vectors part[pb][0..len) in rank order into out[]
  auto cluster_sum = [&](int len, T* out) {
    cl.sync();
    for (int e = tid; e < len; e += blockDim.x) {
      T s = zero<T>();
      for (int q0 = 0; q0 < Q; q0 += 8) {
        T v[8];   // eight remote loads issued together, then added in rank order
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q0 + q < Q) v[q] = cl.map_shared_rank(part + pb * pst, q0 + q)[e];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q0 + q < Q) s = s + v[q];
      }
      out[e] = s;
    }
    pb ^= 1;
    __syncthreads();
  };

  if (tid == 0) {
    int cnt = 0, off = 0;
    for (int dy = -2; dy <= 2; ++dy)
      for (int dx = -2; dx <= 2; ++dx) {
        if (max(abs(dx), abs(dy)) != 2) continue;
        const int mb = nbr_box(B, g, dx, dy);
        if (mb < 0) continue;
        Mbox[cnt] = mb;
        Moff[cnt] = off;
        off += L.nact[mb];
        ++cnt;
      }
    Moff[cnt] = off;
    s_nM = cnt;
  }
  __syncthreads();
  const int nM = s_nM, mh = Moff[nM], P = a.P;
  const int m = a.half ? mh + P : 2 * (mh + P);
  const int r0 = min(m, rank * rp), r1 = min(m, r0 + rp);
  const int bx = B % g, by = B / g;
  const double cx = a.geo.x0 - 0.5 * a.geo.hg + (bx + 0.5) * a.Lbox;
  const double cy = a.geo.y0 - 0.5 * a.geo.hg + (by + 0.5) * a.Lbox;
  // owned rows of Y
  const int mr = r1 - r0;
  for (long long e = tid; e < (long long)mr * n; e += blockDim.x) {
    const int i = r0 + (int)(e % mr), j = (int)(e / mr);
    Yw[(size_t)j * ldY + i] = id_entry(a, B, i, j, mh, Mbox, Moff, cx, cy);
  }
  __syncthreads();
  // column norms: partials over owned rows, summed across the cluster
  for (int c = warp; c < n; c += nwarp) {
    double s = 0.0;
    for (int i = r0 + lane; i < r1; i += 32) s += abs2(Y[(size_t)c * ldY + i]);
    s = warp_sum(s);
    if (lane == 0) part[pb * pst + c] = from_re<T>(s);
  }
  cluster_sum(n, u);   // (u used as scratch)
  for (int c = tid; c < n; c += blockDim.x) {
    norms2[c] = re(u[c]);
    ref[c] = norms2[c];
    perm[c] = c;
  }
  __syncthreads();
  if (warp == 0) {
    double s = 0.0, mx = 0.0;
    for (int c = lane; c < n; c += 32) {
      s += norms2[c];
      mx = fmax(mx, norms2[c]);
    }
    s = warp_sum(s);
    mx = warp_max(mx);
    if (lane == 0) {
      s_thresh = a.eps * a.eps * s;
      s_y2max = mx;
    }
  }
  __syncthreads();

  int k = 0;
  const int kmax = min(m, n);
  while (k < kmax) {
    if (warp == 0) {   // stop test and pivot (identical in every CTA)
      double s = 0.0, mx = -1.0;
      for (int c = k + lane; c < n; c += 32) {
        s += norms2[c];
        mx = fmax(mx, norms2[c]);
      }
      s = warp_sum(s);
      mx = warp_max(mx);
      const double thr = mx - (TIE_REL * mx + TIE_ABS * sqrt(mx * s_y2max));
      int bp = INT_MAX, bc = -1;
      for (int c = k + lane; c < n; c += 32)
        if (norms2[c] >= thr && perm[c] < bp) {
          bp = perm[c];
          bc = c;
        }
      for (int d = 16; d > 0; d >>= 1) {
        const int op = __shfl_xor_sync(0xffffffffu, bp, d), oc = __shfl_xor_sync(0xffffffffu, bc, d);
        if (op < bp) {
          bp = op;
          bc = oc;
        }
      }
      if (lane == 0) {
        s_stop = (s <= s_thresh) || bc < 0;
        if (!s_stop && bc != k) {
          int ti = perm[k]; perm[k] = perm[bc]; perm[bc] = ti;
          double td = norms2[k]; norms2[k] = norms2[bc]; norms2[bc] = td;
          td = ref[k]; ref[k] = ref[bc]; ref[bc] = td;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int q = perm[k];
    // owned rows of the pivot column after k reflectors; partial norm and x0
    double s2 = 0.0;
    for (int i = max(k, r0) + tid; i < r1; i += blockDim.x) {
      T x = Y[(size_t)q * ldY + i];
      for (int l = 0; l < k; ++l) x = msb(x, V[(size_t)l * ldY + i], G[(size_t)l * nmax + q]);
      vbuf[i - r0] = x;
      s2 += abs2(x);
    }
    s2 = warp_sum(s2);
    if (lane == 0) part[pb * pst + 2 + warp] = from_re<T>(s2);
    if (tid == 0) part[pb * pst + 0] = zero<T>();
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < nwarp; ++w) t += re(part[pb * pst + 2 + w]);
      part[pb * pst + 0] = from_re<T>(t);
      part[pb * pst + 1] = (k >= r0 && k < r1) ? vbuf[k - r0] : zero<T>();
    }
    cluster_sum(2, u + nmax - 2);   // u[nmax-2] = alpha^2, u[nmax-1] = x0
    if (tid == 0) {
      const T x0 = u[nmax - 1];
      const double alpha = sqrt(re(u[nmax - 2]));
      if (alpha == 0.0) {
        s_stop = 1;
      } else {
        const double ax0 = sqrt(abs2(x0));
        T phase = from_re<T>(1.0);
        if (ax0 != 0.0) phase = scl(1.0 / ax0, x0);
        const T bt = scl(-alpha, phase);
        beta[k] = bt;
        s_scale = dv(from_re<T>(1.0), x0 - bt);   // 1 / (x0 - beta), one division
        taus[k] = (alpha + ax0) / alpha;
      }
    }
    __syncthreads();
    if (s_stop) break;
    {
      const T d = s_scale;
      for (int i = max(k + 1, r0) + tid; i < r1; i += blockDim.x) {
        const T v = vbuf[i - r0] * d;
        vbuf[i - r0] = v;
        V[(size_t)k * ldY + i] = v;
      }
      if (tid == 0 && k >= r0 && k < r1) {
        vbuf[k - r0] = from_re<T>(1.0);
        V[(size_t)k * ldY + k] = from_re<T>(1.0);
      }
    }
    __syncthreads();
    // partials of u_l = v^H V[:, l] (l < k) and g_c = v^H Y[:, c] over owned rows
    const int nc = n - k - 1;
    const int ib = max(k, r0);
    for (int w = warp; w < k + nc; w += nwarp) {
      const T* col = w < k ? V + (size_t)w * ldY : Y + (size_t)perm[k + 1 + (w - k)] * ldY;
      T d0 = zero<T>(), d1 = zero<T>(), d2 = zero<T>(), d3 = zero<T>();
      int i = ib + lane;
      for (; i + 96 < r1; i += 128) {
        d0 = madc(d0, vbuf[i - r0], col[i]);
        d1 = madc(d1, vbuf[i + 32 - r0], col[i + 32]);
        d2 = madc(d2, vbuf[i + 64 - r0], col[i + 64]);
        d3 = madc(d3, vbuf[i + 96 - r0], col[i + 96]);
      }
      for (; i < r1; i += 32) d0 = madc(d0, vbuf[i - r0], col[i]);
      const T d = warp_sum((d0 + d1) + (d2 + d3));
      if (lane == 0) part[pb * pst + w] = d;
    }
    if (a.g_sm)   // row k of V may belong to another CTA: read through L2
      for (int l = tid; l <= k; l += blockDim.x) vrow[l] = ld_l2(V + (size_t)l * ldY + k);
    cluster_sum(k + nc, u);   // u[0..k): v^H V, u[k..k+nc): raw g for positions k+1..
    // g_c, row k of R, norm downdate (identical in every CTA; own copies of G, Rr)
    const double tau = taus[k];
    int anyf = 0;
    for (int pos = k + 1 + tid; pos < n; pos += blockDim.x) {
      const int c = perm[pos];
      T gc = u[k + (pos - k - 1)];
      for (int l = 0; l < k; ++l) gc = msb(gc, G[(size_t)l * nmax + c], u[l]);
      gc = scl(tau, gc);
      G[(size_t)k * nmax + c] = gc;
      T r = ld_l2(Y + (size_t)c * ldY + k);   // row k may belong to another CTA
      if (a.g_sm)
        for (int l = 0; l <= k; ++l) r = msb(r, vrow[l], G[(size_t)l * nmax + c]);
      else
        for (int l = 0; l <= k; ++l) r = msb(r, ld_l2(V + (size_t)l * ldY + k), G[(size_t)l * nmax + c]);
      Rr[(size_t)k * nmax + c] = r;
      const double nv = norms2[pos] - abs2(r);
      flag[pos] = nv < RECOMPUTE_REL * ref[pos];
      anyf |= flag[pos];
      norms2[pos] = nv;
    }
    // the flags are the same in every CTA of the cluster (same data, same
    // operations), so all of them skip the re-accumulation together
    if (!__syncthreads_or(anyf)) {
      ++k;
      continue;
    }
    // re-accumulation of flagged norms: partials over owned rows
    for (int pos = k + 1 + warp; pos < n; pos += nwarp) {
      double t = 0.0;
      if (flag[pos]) {
        const int c = perm[pos];
        for (int i = max(k + 1, r0) + lane; i < r1; i += 32) {
          T x = Y[(size_t)c * ldY + i];
          for (int l = 0; l <= k; ++l) x = msb(x, V[(size_t)l * ldY + i], G[(size_t)l * nmax + c]);
          t += abs2(x);
        }
        t = warp_sum(t);
      }
      if (lane == 0) part[pb * pst + pos] = from_re<T>(t);
    }
    cluster_sum(n, u);
    for (int pos = k + 1 + tid; pos < n; pos += blockDim.x)
      if (flag[pos]) {
        norms2[pos] = re(u[pos]);
        ref[pos] = norms2[pos];
      }
    __syncthreads();
    ++k;
  }
  cl.sync();   // every CTA is done reading its peers' shared memory
  if (rank != 0) return;
  // T = R11^{-1} R12 (back substitution), k x r with ld nmax
  const int r = n - k;
  S* Tw = a.T_ws + (size_t)bi * nn;
  for (int c = tid; c < r; c += blockDim.x) {
    const int oc = perm[k + c];
    for (int i = k - 1; i >= 0; --i) {
      T x = Rr[(size_t)i * nmax + oc];
      for (int l = i + 1; l < k; ++l)
        x = msb(x, Rr[(size_t)i * nmax + perm[l]], id_load<T, S>(Tw[(size_t)c * nmax + l]));
      Tw[(size_t)c * nmax + i] = id_store<T, S>(dv(x, beta[i]));
    }
  }
  for (int c = tid; c < n; c += blockDim.x) a.perm_out[(size_t)bi * nmax + c] = perm[c];
  if (tid == 0) a.k_out[bi] = k;
}

// ------------------------------------------------------------------ tensor-core helpers

// ------------------------------------------------------------------ digit slices
// A row x_0..x_{r-1} with max |x_l| = m 2^e (m in [0.5, 1)) is written as
// x_l = 2^e sum_{p=0}^{OZ_S-1} d_{p,l} 2^{-7(p+1)}, with signed digits
// |d_0| <= 128 and |d_p| <= 64 (p >= 1), all exact in bf16; the truncation error
// is below 2^(e-57), the rounding of x 2^(56-e) to an integer.
__device__ inline uint16_t bf16_of_small_int(int d) {
  const __nv_bfloat16 h = __float2bfloat16_rn((float)d);
  return __bfloat16_as_ushort(h);
}

__device__ void oz_split_row(const double* __restrict__ src, int stride, int r, int kp, uint16_t* dst, int* eout) {
  double mx = 0.0;
  for (int l = 0; l < r; ++l) mx = fmax(mx, fabs(src[(size_t)l * stride]));
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);
  *eout = e;
  const double scale = ldexp(1.0, 56 - e);
  for (int l = 0; l < kp; l += 2) {
    long long X0 = l < r ? llrint(src[(size_t)l * stride] * scale) : 0;
    long long X1 = l + 1 < r ? llrint(src[(size_t)(l + 1) * stride] * scale) : 0;
    int d0[OZ_S], d1[OZ_S];
#pragma unroll
    for (int p = OZ_S - 1; p >= 1; --p) {
      d0[p] = (int)(((X0 + 64) & 127) - 64);
      X0 = (X0 - d0[p]) >> OZ_BITS;
      d1[p] = (int)(((X1 + 64) & 127) - 64);
      X1 = (X1 - d1[p]) >> OZ_BITS;
    }
    d0[0] = (int)X0;
    d1[0] = (int)X1;
#pragma unroll
    for (int p = 0; p < OZ_S; ++p)
      *reinterpret_cast<uint32_t*>(dst + (size_t)p * kp + l) =
          (uint32_t)bf16_of_small_int(d0[p]) | ((uint32_t)bf16_of_small_int(d1[p]) << 16);
  }
}

// ------------------------------------------------------------------ sparsify + LU (Eqs. 7, 8)
template <typename T> struct ElimArgs {
  LevelDev<T> L;
  const BoxRec<T>* recs;
  const int* cls_idx;       // class index of each record's box (row into perm/T_ws)
  const int* perm_in;
  const T* T_ws;
  int* err;
  int smem_cap;             // scalars of dynamic shared memory available
  int sym;                  // A is symmetric (real Laplace): A_BC^T = A_CB
};

constexpr int PKC = 16;     // rows of a panel product's right operand staged per chunk

// Register-blocked panel product: out(i, j) = init(i, j) + sum_l A_l[i] B(l, j)
// for the rows i < rows of a panel of 16 MA rows and the columns j of the block
// [j0, min(r, j0 + 16 NB)).  arow(l) points at row l of the left operand (16 MA
// scalars in shared memory); B(l, j) is read through bfun in chunks of PKC rows
// staged in Bs (PKC x (16 NB + 1)).  Thread (tx, ty) owns rows tx + 16 a and
// columns j0 + ty + 16 b.  TRI: B is upper triangular (B(l, j) = 0 for l > j).
// Every thread of the block calls it; out() runs after a barrier, so it may
// overwrite what init() reads.
template <typename T, int MA, int NB, bool TRI, typename AR, typename BF, typename IF, typename OF>
__device__ __forceinline__ void panel_gemm(AR arow, int nl, int rows, int j0, int r, T* Bs, BF bfun, IF init,
                                           OF out) {
  constexpr int RB = 16 * NB + 1;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[MA][NB];
#pragma unroll
  for (int a = 0; a < MA; ++a)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int i = tx + 16 * a, j = j0 + ty + 16 * b;
      acc[a][b] = (i < rows && j < r) ? init(i, j) : zero<T>();
    }
  const int jw = min(16 * NB, r - j0);                              // columns in the block
  const int lend = TRI ? min(nl, j0 + jw) : nl;                     // rows of B that can be nonzero
  const int tend = TRI ? min(lend, j0 + ty + 16 * (NB - 1) + 1) : lend;   // this thread's last row
  for (int l0 = 0; l0 < lend; l0 += PKC) {
    __syncthreads();
    for (int e = threadIdx.x; e < PKC * 16 * NB; e += blockDim.x) {
      const int ll = e % PKC, jj = e / PKC, l = l0 + ll, j = j0 + jj;
      Bs[ll * RB + jj] = (l < lend && jj < jw && (!TRI || l <= j)) ? bfun(l, j) : zero<T>();
    }
    __syncthreads();
    const int le = min(PKC, tend - l0);
    for (int ll = 0; ll < le; ++ll) {
      const T* ar = arow(l0 + ll);
      T av[MA], bv[NB];
#pragma unroll
      for (int a = 0; a < MA; ++a) av[a] = ar[tx + 16 * a];
#pragma unroll
      for (int b = 0; b < NB; ++b) bv[b] = Bs[ll * RB + ty + 16 * b];
#pragma unroll
      for (int a = 0; a < MA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[a][b] = mad(acc[a][b], av[a], bv[b]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < MA; ++a)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int i = tx + 16 * a, j = j0 + ty + 16 * b;
      if (i < rows && j < r) out(i, j, acc[a][b]);
    }
}

// Calls f(std::integral_constant<int, NB>) for every 16 NBMAX-column block of
// [0, r), NB = the block's column groups of 16.
template <int NBMAX, typename F> __device__ __forceinline__ void for_col_blocks(int r, F f) {
  for (int j0 = 0; j0 < r; j0 += 16 * NBMAX) {
    const int nb = (min(r - j0, 16 * NBMAX) + 15) / 16;
    switch (nb) {
      case 1: f(j0, std::integral_constant<int, 1>{}); break;
      case 2: if constexpr (NBMAX >= 2) f(j0, std::integral_constant<int, 2>{}); break;
      case 3: if constexpr (NBMAX >= 3) f(j0, std::integral_constant<int, 3>{}); break;
      case 4: if constexpr (NBMAX >= 4) f(j0, std::integral_constant<int, 4>{}); break;
      case 5: if constexpr (NBMAX >= 5) f(j0, std::integral_constant<int, 5>{}); break;
      case 6: if constexpr (NBMAX >= 6) f(j0, std::integral_constant<int, 6>{}); break;
      case 7: if constexpr (NBMAX >= 7) f(j0, std::integral_constant<int, 7>{}); break;
      default: if constexpr (NBMAX >= 8) f(j0, std::integral_constant<int, 8>{}); break;
    }
  }
}

// Complex rows: real and imaginary parts share the row scale (the largest |Re|,
// |Im| of the row) and are split into OZ_S slices each; a row holds the OZ_S
// real slices followed by the OZ_S imaginary slices.
__device__ void oz_split_row(const zd* __restrict__ src, int stride, int r, int kp, uint16_t* dst, int* eout) {
  double mx = 0.0;
  for (int l = 0; l < r; ++l) {
    const zd v = src[(size_t)l * stride];
    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
  }
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);
  *eout = e;
  const double scale = ldexp(1.0, 56 - e);
  for (int part = 0; part < 2; ++part)
    for (int l = 0; l < kp; l += 2) {
      const zd v0 = l < r ? src[(size_t)l * stride] : zd{0.0, 0.0};
      const zd v1 = l + 1 < r ? src[(size_t)(l + 1) * stride] : zd{0.0, 0.0};
      long long X0 = llrint((part ? v0.y : v0.x) * scale);
      long long X1 = llrint((part ? v1.y : v1.x) * scale);
      int d0[OZ_S], d1[OZ_S];
#pragma unroll
      for (int p = OZ_S - 1; p >= 1; --p) {
        d0[p] = (int)(((X0 + 64) & 127) - 64);
        X0 = (X0 - d0[p]) >> OZ_BITS;
        d1[p] = (int)(((X1 + 64) & 127) - 64);
        X1 = (X1 - d1[p]) >> OZ_BITS;
      }
      d0[0] = (int)X0;
      d1[0] = (int)X1;
#pragma unroll
      for (int p = 0; p < OZ_S; ++p)
        *reinterpret_cast<uint32_t*>(dst + (size_t)(part * OZ_S + p) * kp + l) =
            (uint32_t)bf16_of_small_int(d0[p]) | ((uint32_t)bf16_of_small_int(d1[p]) << 16);
    }
}

// LU with partial pivoting of the r x r matrix LU (ld r) by the whole CTA:
// largest modulus, lowest row on ties; the exchanges go to piv.  Returns false
// (after flagging RSS_ENUMERIC) on a zero pivot; piv then holds no exchange for
// the remaining steps, so kernels that still read it index within 0 .. r-1.
template <typename T> __device__ bool lu_pp_block(T* LU, int r, int* piv, int* err) {
  __shared__ int s_piv, s_zero;
  __shared__ __align__(16) double s_dinv[2];   // 1 / pivot, computed once per step (T = double or zd)
  const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (int j = 0; j < r; ++j) {
    if (warp == 0) {
      double mx = -1.0;
      int mi = INT_MAX;
      for (int i = j + lane; i < r; i += 32) {
        const double v = abs2(LU[i + (size_t)j * r]);
        if (v > mx) { mx = v; mi = i; }
      }
      for (int d = 16; d > 0; d >>= 1) {
        const double om = __shfl_xor_sync(0xffffffffu, mx, d);
        const int oi = __shfl_xor_sync(0xffffffffu, mi, d);
        if (om > mx || (om == mx && oi < mi)) { mx = om; mi = oi; }
      }
      if (lane == 0) {
        s_piv = mi;
        s_zero = !(mx > 0.0);
        if (mx > 0.0) *reinterpret_cast<T*>(s_dinv) = dv(from_re<T>(1.0), LU[mi + (size_t)j * r]);
      }
    }
    __syncthreads();
    if (s_zero) {
      if (tid == 0) atomicExch(err, (int)RSS_ENUMERIC);
      for (int i = j + tid; i < r; i += bs) piv[i] = i;
      __syncthreads();
      return false;
    }
    const int p = s_piv;
    if (p != j)
      for (int col = tid; col < r; col += bs) {
        const T t = LU[j + (size_t)col * r];
        LU[j + (size_t)col * r] = LU[p + (size_t)col * r];
        LU[p + (size_t)col * r] = t;
      }
    if (tid == 0) piv[j] = p;
    __syncthreads();
    const T d = *reinterpret_cast<const T*>(s_dinv);
    for (int i = j + 1 + tid; i < r; i += bs) LU[i + (size_t)j * r] = LU[i + (size_t)j * r] * d;
    __syncthreads();
    const int w = r - j - 1;
    for (int e = tid; e < w * w; e += bs) {
      const int ii = j + 1 + e % w, jj = j + 1 + e / w;
      LU[ii + (size_t)jj * r] = msb(LU[ii + (size_t)jj * r], LU[ii + (size_t)j * r], LU[j + (size_t)jj * r]);
    }
    __syncthreads();
  }
  return true;
}

// ------------------------------------------------------------------ sparsify + LU (Eqs. 7, 8)
// k_elim_lu (one CTA per box): C map, X_SR, X_RR, P X_RR = L U, U^{-1}, L^{-1}
// and L^{-1} P.  k_elim_panels (one CTA per 16-, 32- or 64-row panel of C): X_CR, X_RC and
// E = X_CR U^{-1}, F = L^{-1} P X_RC (kept as F^T), from shared-memory panels.
// Boxes too large for the panel kernel's shared memory get E and F here, row by
// row from global memory.
template <typename T> __global__ void __launch_bounds__(NT, 4) k_elim_lu(ElimArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const LevelDev<T>& L = a.L;
  const BoxRec<T> R = a.recs[blockIdx.x];
  const int nmax = L.nmax, g = L.g, B = R.box, k = R.k, r = R.r, c = R.c;
  const size_t nn = (size_t)nmax * nmax;
  const int* perm = a.perm_in + (size_t)a.cls_idx[blockIdx.x] * nmax;
  const T* Tw = a.T_ws + (size_t)a.cls_idx[blockIdx.x] * nn;
  const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, warp = tid >> 5;
  // on chip: LU (r x r), then one region holding T until X_RR is formed and
  // the inverses while they are built
  int* sperm = reinterpret_cast<int*>(smraw);   // 2 r: exchange order and its inverse
  unsigned char* smT = smraw + ((2 * r * sizeof(int) + 15) & ~size_t(15));
  const bool onchip = (size_t)r * r + (size_t)max(k * r, r * r) <= (size_t)a.smem_cap;
  T* LU = onchip ? reinterpret_cast<T*>(smT) : R.LU;
  T* Ts = onchip ? LU + (size_t)r * r : R.Tm;
  T* Wb = onchip ? Ts : nullptr;
  __shared__ int nb[9], coff[10], ord[9];
  if (tid == 0) {
    const int o9[9] = {4, 0, 1, 2, 3, 5, 6, 7, 8};
    int off = 0;
    for (int q = 0; q < 9; ++q) {
      const int s = o9[q];
      ord[q] = s;
      nb[s] = nbr_box(B, g, s % 3 - 1, s / 3 - 1);
      coff[q] = off;
      off += s == 4 ? k : (nb[s] >= 0 ? L.nact[nb[s]] : 0);
    }
    coff[9] = off;
  }
  __syncthreads();
  for (int i = tid; i < c; i += bs) {
    int q = 0;
    while (coff[q + 1] <= i) ++q;
    const int s = ord[q], ii = i - coff[q], u = nb[s];
    const int pos = s == 4 ? perm[ii] : L.act[u * nmax + ii];
    R.cmap[i] = (s << 16) | pos;
    R.idxC[i] = L.pts[u * nmax + pos];
  }
  for (int j = tid; j < r; j += bs) R.idxR[j] = L.pts[B * nmax + perm[k + j]];
  for (int e = tid; e < k * r; e += bs) {
    const T t = Tw[(size_t)(e / k) * nmax + e % k];
    R.Tm[e] = t;
    if (onchip) Ts[e] = t;
  }
  __syncthreads();
  const T* Abb = L.blk + ((size_t)B * 25 + 12) * nn;
  // X_SR = A_SR - A_SS T into E's first k rows (the rows of S in C)
  for (int e = tid; e < k * r; e += bs) {
    const int si = e % k, j = e / k;
    T x = Abb[(size_t)perm[k + j] * nmax + perm[si]];
    for (int q = 0; q < k; ++q) x = msb(x, Abb[(size_t)perm[q] * nmax + perm[si]], Ts[q + (size_t)j * k]);
    R.E[si + (size_t)j * c] = x;
  }
  __syncthreads();
  // X_RR = A_RR - A_RS T - T^* X_SR
  for (int e = tid; e < r * r; e += bs) {
    const int ai = e % r, bj = e / r;
    T x = Abb[(size_t)perm[k + bj] * nmax + perm[k + ai]];
    for (int q = 0; q < k; ++q) x = msb(x, Abb[(size_t)perm[q] * nmax + perm[k + ai]], Ts[q + (size_t)bj * k]);
    for (int q = 0; q < k; ++q) x = msbc(x, Ts[q + (size_t)ai * k], R.E[q + (size_t)bj * c]);
    LU[ai + (size_t)bj * r] = x;
  }
  __syncthreads();
  // P X_RR = L U, partial pivoting (largest modulus, lowest row on ties)   (Eq. 8)
  if (!lu_pp_block(LU, r, R.piv, a.err)) return;
  // U^{-1} and L^{-1}, one column per thread (built in shared memory when it
  // fits, then copied out); L^{-1} P is L^{-1} with its columns permuted:
  // P e_j = e_{pos(j)} for pos the inverse of the exchange order sig (P v = v[sig])
  for (int which = 0; which < 2; ++which) {
    T* dst = which == 0 ? R.Ui : R.Li;
    T* W = onchip ? Wb : dst;
    for (int j = tid; j < r; j += bs) {
      T* w = W + (size_t)j * r;
      if (which == 0) {               // U^{-1} e_j
        for (int i = j + 1; i < r; ++i) w[i] = zero<T>();
        for (int i = j; i >= 0; --i) {
          T x = i == j ? from_re<T>(1.0) : zero<T>();
          for (int l = i + 1; l <= j; ++l) x = msb(x, LU[i + (size_t)l * r], w[l]);
          w[i] = dv(x, LU[i + (size_t)i * r]);
        }
      } else {                        // L^{-1} e_j
        for (int i = 0; i < j; ++i) w[i] = zero<T>();
        w[j] = from_re<T>(1.0);
        for (int i = j + 1; i < r; ++i) {
          T x = zero<T>();
          for (int l = j; l < i; ++l) x = msb(x, LU[i + (size_t)l * r], w[l]);
          w[i] = x;
        }
      }
    }
    __syncthreads();
    if (onchip)
      for (int e = tid; e < r * r; e += bs) dst[e] = Wb[e];
    if (which == 1) {
      if (tid == 0) {
        for (int i = 0; i < r; ++i) sperm[i] = i;
        for (int i = 0; i < r; ++i) {
          const int p = R.piv[i], t = sperm[i];
          sperm[i] = sperm[p];
          sperm[p] = t;
        }
        for (int i = 0; i < r; ++i) sperm[r + sperm[i]] = i;
      }
      __syncthreads();
      for (int e = tid; e < r * r; e += bs) {
        const int i = e % r, j = e / r;
        R.LiP[e] = W[i + (size_t)sperm[r + j] * r];
      }
    }
    __syncthreads();
  }
  if (onchip)
    for (int e = tid; e < r * r; e += bs) R.LU[e] = LU[e];
  __syncthreads();
  if (R.ozp) {
    // W_E = [-T U^{-1}; U^{-1}] and W_F = [-(L^{-1} P T^*)^T; (L^{-1} P)^T], n x r, ld n:
    // E = X_CR U^{-1} = A_CB W_E and F^T = (L^{-1} P X_RC)^T = A_BC^T W_F (Eqs. 7, 8)
    const int n = k + r;
    for (int e = tid; e < n * r; e += bs) {
      const int l = e % n, j = e / n;
      T we, wf;
      if (l < k) {
        we = zero<T>();
        for (int m = 0; m <= j; ++m) we = msb(we, R.Tm[l + (size_t)m * k], R.Ui[m + (size_t)j * r]);
        wf = zero<T>();
        for (int m = 0; m < r; ++m) wf = msb(wf, R.LiP[j + (size_t)m * r], cj(R.Tm[l + (size_t)m * k]));
      } else {
        we = l - k <= j ? R.Ui[(l - k) + (size_t)j * r] : zero<T>();
        wf = R.LiP[j + (size_t)(l - k) * r];
      }
      R.We[e] = we;
      R.Wf[e] = wf;
    }
  }
  if (!R.panels && !R.ozp) {
    // E and F^T row by row from global memory
    for (long long e = tid; e < (long long)c * r; e += bs) {
      const int i = (int)(e % c), j = (int)(e / c);
      const int cm = R.cmap[i], s = cm >> 16, pos = cm & 0xffff, u = nb[s];
      const T* Aub = L.blk + ((size_t)u * 25 + off_index(u, B, g)) * nn;
      const T* Abu = L.blk + ((size_t)B * 25 + off_index(B, u, g)) * nn;
      const int rj = perm[k + j];
      T x = Aub[(size_t)rj * nmax + pos];
      T y = Abu[(size_t)pos * nmax + rj];
      for (int q = 0; q < k; ++q) {
        const T t = R.Tm[q + (size_t)j * k];
        x = msb(x, Aub[(size_t)perm[q] * nmax + pos], t);
        y = msbc(y, t, Abu[(size_t)pos * nmax + perm[q]]);
      }
      R.E[i + (size_t)j * c] = x;
      R.Ft[i + (size_t)j * c] = y;
    }
    __syncthreads();
    for (int i = tid; i < c; i += bs) {
      T* e = R.E + i;
      for (int j = r - 1; j >= 0; --j) {
        T x = zero<T>();
        for (int l = 0; l <= j; ++l) x = mad(x, e[(size_t)l * c], R.Ui[l + (size_t)j * r]);
        e[(size_t)j * c] = x;
      }
      T* f = R.Ft + i;
      for (int j = 0; j < r; ++j) {
        const int p = R.piv[j];
        if (p != j) {
          const T t = f[(size_t)j * c];
          f[(size_t)j * c] = f[(size_t)p * c];
          f[(size_t)p * c] = t;
        }
      }
      for (int j = 1; j < r; ++j) {
        T x = f[(size_t)j * c];
        for (int l = 0; l < j; ++l) x = msb(x, R.LU[j + (size_t)l * r], f[(size_t)l * c]);
        f[(size_t)j * c] = x;
      }
    }
    __syncthreads();
    if (R.Esl != nullptr) {
      const int ns = sizeof(T) == sizeof(double) ? OZ_S : 2 * OZ_S;   // slices per row
      for (int i = tid; i < 2 * c; i += bs) {
        const bool isE = i < c;
        const int row = isE ? i : i - c;
        oz_split_row((isE ? R.E : R.Ft) + row, c, r, R.kp,
                     (isE ? R.Esl : R.Fsl) + (size_t)row * ns * R.kp, (isE ? R.Eexp : R.Fexp) + row);
      }
    }
  }
  // B keeps only its skeleton
  for (int q = tid; q < k; q += bs) L.act[B * nmax + q] = perm[q];
  if (tid == 0) L.nact[B] = k;
}

// One panel of 16 MA rows of C.  The rows of A(u, B) (columns of B in pivot
// order) sit in shared memory as [column][row]; X_CR overwrites the R columns in
// place, then E = X_CR U^{-1} goes to global memory; the same buffer then takes
// the columns of A(B, u) for X_RC and F^T = (L^{-1} P_R X_RC)^T.  The right
// operands (T, U^{-1}, L^{-1}) are staged from global memory in chunks, so any
// rank fits.
// On-chip k_elim_lu for boxes whose blocks fit in shared memory (and whose E
// and F come from the panel kernels): the permuted diagonal block A_BB is
// staged by cp.async, and X_SR, X_RR, the LU and both triangular inverses stay
// on chip.  Every phase spreads its work over the whole CTA; U^{-1} and L^{-1}
// are built by row sweeps (after row i is final it is subtracted from the
// rows it feeds, one rank-1 update per row).
template <typename T> __host__ __device__ inline size_t elim_lu_sm_bytes(int k, int r) {
  const size_t n = (size_t)k + r;
  const size_t ints = ((n + 2 * (size_t)r) * sizeof(int) + 15) & ~size_t(15);
  const size_t kr = (size_t)k * r, rr = (size_t)r * r;
  return ints + sizeof(T) * (n * n + kr + (kr > rr ? kr : rr) + rr + r);
}

template <typename T> __global__ void __launch_bounds__(NT, 2) k_elim_lu_sm(ElimArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const LevelDev<T>& L = a.L;
  const BoxRec<T> R = a.recs[blockIdx.x];
  const int nmax = L.nmax, g = L.g, B = R.box, k = R.k, r = R.r, c = R.c, n = k + r;
  const size_t nn = (size_t)nmax * nmax;
  const int* perm_g = a.perm_in + (size_t)a.cls_idx[blockIdx.x] * nmax;
  const T* Tw = a.T_ws + (size_t)a.cls_idx[blockIdx.x] * nn;
  const int tid = threadIdx.x, bs = blockDim.x;
  int* sp = reinterpret_cast<int*>(smraw);   // n: B's points in pivot order
  int* sperm = sp + n;                      // 2 r: exchange order and its inverse
  T* Ap = reinterpret_cast<T*>(smraw + (((size_t)(n + 2 * r) * sizeof(int) + 15) & ~size_t(15)));   // n x n
  T* Ts = Ap + (size_t)n * n;                       // k x r
  T* Xs = Ts + (size_t)k * r;                       // k x r: X_SR; later U^{-1} (r x r)
  T* LU = Xs + (size_t)max(k * r, r * r);           // r x r, then r reciprocals of U's diagonal
  T* Ui = Xs;
  T* Li = Ap;                                       // r x r, once A_BB is no longer needed
  __shared__ int nb[9], coff[10], ord[9];
  if (tid == 0) {
    const int o9[9] = {4, 0, 1, 2, 3, 5, 6, 7, 8};
    int off = 0;
    for (int q = 0; q < 9; ++q) {
      const int s = o9[q];
      ord[q] = s;
      nb[s] = nbr_box(B, g, s % 3 - 1, s / 3 - 1);
      coff[q] = off;
      off += s == 4 ? k : (nb[s] >= 0 ? L.nact[nb[s]] : 0);
    }
    coff[9] = off;
  }
  for (int i = tid; i < n; i += bs) sp[i] = perm_g[i];
  __syncthreads();
  const T* Abb = L.blk + ((size_t)B * 25 + 12) * nn;
  for (int e = tid; e < n * n; e += bs) cp_async_el(Ap + e, Abb + (size_t)sp[e / n] * nmax + sp[e % n]);
  for (int e = tid; e < k * r; e += bs) cp_async_el(Ts + e, Tw + (size_t)(e / k) * nmax + e % k);
  for (int i = tid; i < c; i += bs) {
    int q = 0;
    while (coff[q + 1] <= i) ++q;
    const int s = ord[q], ii = i - coff[q], u = nb[s];
    const int pos = s == 4 ? sp[ii] : L.act[u * nmax + ii];
    R.cmap[i] = (s << 16) | pos;
    R.idxC[i] = L.pts[u * nmax + pos];
  }
  for (int j = tid; j < r; j += bs) R.idxR[j] = L.pts[B * nmax + sp[k + j]];
  cp_async_wait_all();
  __syncthreads();
  for (int e = tid; e < k * r; e += bs) R.Tm[e] = Ts[e];
  // X_SR = A_SR - A_SS T
  for (int e = tid; e < k * r; e += bs) {
    const int si = e % k, j = e / k;
    T x = Ap[si + (size_t)(k + j) * n];
    for (int q = 0; q < k; ++q) x = msb(x, Ap[si + (size_t)q * n], Ts[q + (size_t)j * k]);
    Xs[e] = x;
  }
  __syncthreads();
  // X_RR = A_RR - A_RS T - T^* X_SR
  for (int e = tid; e < r * r; e += bs) {
    const int ai = e % r, bj = e / r;
    T x = Ap[(k + ai) + (size_t)(k + bj) * n];
    for (int q = 0; q < k; ++q) x = msb(x, Ap[(k + ai) + (size_t)q * n], Ts[q + (size_t)bj * k]);
    for (int q = 0; q < k; ++q) x = msbc(x, Ts[q + (size_t)ai * k], Xs[q + (size_t)bj * k]);
    LU[e] = x;
  }
  __syncthreads();
  if (!lu_pp_block(LU, r, R.piv, a.err)) return;
  // U^{-1}: rows from the bottom
  for (int e = tid; e < r * r; e += bs) Ui[e] = (e % r == e / r) ? from_re<T>(1.0) : zero<T>();
  for (int e = tid; e < r * r; e += bs) Li[e] = (e % r == e / r) ? from_re<T>(1.0) : zero<T>();
  T* Dr = LU + (size_t)r * r;   // r reciprocals of the diagonal of U, one division each
  for (int i = tid; i < r; i += bs) Dr[i] = dv(from_re<T>(1.0), LU[i + (size_t)i * r]);
  __syncthreads();
  for (int i = r - 1; i >= 0; --i) {
    const T d = Dr[i];
    for (int j = i + tid; j < r; j += bs) Ui[i + (size_t)j * r] = Ui[i + (size_t)j * r] * d;
    __syncthreads();
    const int w = r - i;
    for (int e = tid; e < i * w; e += bs) {
      const int l = e % i, j = i + e / i;
      Ui[l + (size_t)j * r] = msb(Ui[l + (size_t)j * r], LU[l + (size_t)i * r], Ui[i + (size_t)j * r]);
    }
    __syncthreads();
  }
  // L^{-1} (unit lower): rows from the top
  for (int i = 0; i < r - 1; ++i) {
    const int below = r - 1 - i;
    for (int e = tid; e < below * (i + 1); e += bs) {
      const int l = i + 1 + e % below, j = e / below;
      Li[l + (size_t)j * r] = msb(Li[l + (size_t)j * r], LU[l + (size_t)i * r], Li[i + (size_t)j * r]);
    }
    __syncthreads();
  }
  if (tid == 0) {   // exchange order sig (P v = v[sig]) and its inverse
    for (int i = 0; i < r; ++i) sperm[i] = i;
    for (int i = 0; i < r; ++i) {
      const int p = R.piv[i], t = sperm[i];
      sperm[i] = sperm[p];
      sperm[p] = t;
    }
    for (int i = 0; i < r; ++i) sperm[r + sperm[i]] = i;
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += bs) {
    R.LU[e] = LU[e];
    R.Ui[e] = Ui[e];
    R.Li[e] = Li[e];
    R.LiP[e] = Li[e % r + (size_t)sperm[r + e / r] * r];
  }
  if (R.ozp) {   // W_E and W_F, as in k_elim_lu
    for (int e = tid; e < n * r; e += bs) {
      const int l = e % n, j = e / n;
      T we, wf;
      if (l < k) {
        we = zero<T>();
        for (int m = 0; m <= j; ++m) we = msb(we, Ts[l + (size_t)m * k], Ui[m + (size_t)j * r]);
        wf = zero<T>();
        for (int m = 0; m < r; ++m) wf = msb(wf, Li[j + (size_t)sperm[r + m] * r], cj(Ts[l + (size_t)m * k]));
      } else {
        we = l - k <= j ? Ui[(l - k) + (size_t)j * r] : zero<T>();
        wf = Li[j + (size_t)sperm[r + l - k] * r];
      }
      R.We[e] = we;
      R.Wf[e] = wf;
    }
  }
  // B keeps only its skeleton
  for (int q = tid; q < k; q += bs) L.act[B * nmax + q] = sp[q];
  if (tid == 0) L.nact[B] = k;
}

template <typename T, int MA, int NBMAX>
__device__ void elim_panel_body(const ElimArgs<T>& a, const BoxRec<T>& R, unsigned char* smraw, int p0, int rows) {
  constexpr int EPR = 16 * MA;
  const LevelDev<T>& L = a.L;
  const int nmax = L.nmax, g = L.g, B = R.box, k = R.k, r = R.r, c = R.c, n = k + r;
  const size_t nn = (size_t)nmax * nmax;
  const int* perm = a.perm_in + (size_t)a.cls_idx[blockIdx.y] * nmax;
  const int tid = threadIdx.x, bs = blockDim.x;
  T* As = reinterpret_cast<T*>(smraw);                 // n x EPR
  T* Bs = As + (size_t)n * EPR;                        // PKC x (16 NBMAX + 1)
  int* sig = reinterpret_cast<int*>(Bs + PKC * (16 * NBMAX + 1));   // r
  const T* __restrict__ Tm = R.Tm;
  const T* __restrict__ Ui = R.Ui;
  const T* __restrict__ Li = R.Li;
  for (int e = tid; e < rows * n; e += bs) {   // rows of A(u, B), columns of B in pivot order
    const int ii = e % rows, col = e / rows;
    const int cm = R.cmap[p0 + ii], s = cm >> 16, pos = cm & 0xffff;
    const int u = nbr_box(B, g, s % 3 - 1, s / 3 - 1);
    As[col * EPR + ii] = L.blk[((size_t)u * 25 + off_index(u, B, g)) * nn + (size_t)perm[col] * nmax + pos];
  }
  if (tid == 0) {   // P_R v = v[sig]: the row exchanges applied to the identity
    for (int i = 0; i < r; ++i) sig[i] = i;
    for (int i = 0; i < r; ++i) {
      const int p = R.piv[i], t = sig[i];
      sig[i] = sig[p];
      sig[p] = t;
    }
  }
  __syncthreads();
  auto plain = [&](int l) { return As + (size_t)l * EPR; };
  auto rcol = [&](int l) { return As + (size_t)(k + l) * EPR; };
  // X_CR = A_CR - A_CS T, in place
  for_col_blocks<NBMAX>(r, [&](int j0, auto nbc) {
    panel_gemm<T, MA, decltype(nbc)::value, false>(
        plain, k, rows, j0, r, Bs, [&](int q, int j) { return -Tm[q + (size_t)j * k]; },
        [&](int i, int j) { return As[(k + j) * EPR + i]; }, [&](int i, int j, T v) { As[(k + j) * EPR + i] = v; });
  });
  // E = X_CR U^{-1}
  for_col_blocks<NBMAX>(r, [&](int j0, auto nbc) {
    panel_gemm<T, MA, decltype(nbc)::value, true>(
        rcol, r, rows, j0, r, Bs, [&](int l, int j) { return Ui[l + (size_t)j * r]; },
        [&](int, int) { return zero<T>(); }, [&](int i, int j, T v) { R.E[p0 + i + (size_t)j * c] = v; });
  });
  __syncthreads();
  for (int e = tid; e < rows * n; e += bs) {   // columns of A(B, u), rows of B in pivot order
    const int row = e % n, ii = e / n;
    const int cm = R.cmap[p0 + ii], s = cm >> 16, pos = cm & 0xffff;
    const int u = nbr_box(B, g, s % 3 - 1, s / 3 - 1);
    As[row * EPR + ii] = L.blk[((size_t)B * 25 + off_index(B, u, g)) * nn + (size_t)pos * nmax + perm[row]];
  }
  __syncthreads();
  // X_RC^T = A_RC^T - A_SC^T conj(T), in place
  for_col_blocks<NBMAX>(r, [&](int j0, auto nbc) {
    panel_gemm<T, MA, decltype(nbc)::value, false>(
        plain, k, rows, j0, r, Bs, [&](int q, int j) { return -cj(Tm[q + (size_t)j * k]); },
        [&](int i, int j) { return As[(k + j) * EPR + i]; }, [&](int i, int j, T v) { As[(k + j) * EPR + i] = v; });
  });
  // F^T = (P_R X_RC)^T (L_R^{-1})^T: row l of P_R X_RC is row sig[l] of X_RC;
  // (L^{-1})^T is upper triangular
  auto prow = [&](int l) { return As + (size_t)(k + sig[l]) * EPR; };
  for_col_blocks<NBMAX>(r, [&](int j0, auto nbc) {
    panel_gemm<T, MA, decltype(nbc)::value, true>(
        prow, r, rows, j0, r, Bs, [&](int l, int j) { return Li[j + (size_t)l * r]; },
        [&](int, int) { return zero<T>(); }, [&](int i, int j, T v) { R.Ft[p0 + i + (size_t)j * c] = v; });
  });
  __syncthreads();
  if (R.Esl != nullptr) {   // digit slices of this panel's rows of E and F^T
    const int ns = sizeof(T) == sizeof(double) ? OZ_S : 2 * OZ_S;
    for (int e = tid; e < 2 * rows; e += bs) {
      const bool isE = e < rows;
      const int row = p0 + (isE ? e : e - rows);
      oz_split_row((isE ? R.E : R.Ft) + row, c, r, R.kp,
                   (isE ? R.Esl : R.Fsl) + (size_t)row * ns * R.kp, (isE ? R.Eexp : R.Fexp) + row);
    }
  }
}

template <typename T> constexpr int panel_nbmax() { return sizeof(T) == sizeof(double) ? 6 : 4; }

// shared memory of one panel CTA of 16 MA rows for a box with n = k + r points
template <typename T> size_t panel_smem_bytes(int MA, int n, int r) {
  return sizeof(T) * ((size_t)n * 16 * MA + (size_t)PKC * (16 * panel_nbmax<T>() + 1)) + sizeof(int) * (size_t)r;
}

template <typename T, int MA> __global__ void __launch_bounds__(NT, 2) k_elim_panels(ElimArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BoxRec<T> R = a.recs[blockIdx.y];
  if (!R.panels || R.ozp) return;
  const int p0 = blockIdx.x * 16 * MA;
  if (p0 >= R.c) return;
  elim_panel_body<T, MA, panel_nbmax<T>()>(a, R, smraw, p0, min(16 * MA, R.c - p0));
}


// Real factors: the columns of W_E and W_F cut into digit slices once per box
// (every panel CTA of the box reads them).  One CTA per box, eight threads per
// column.
__global__ void __launch_bounds__(NT) k_w_split(ElimArgs<double> a) {
  const BoxRec<double> R = a.recs[blockIdx.x];
  if (!R.ozp) return;
  const int r = R.r, n = R.k + r, np = (n + 15) & ~15, rp = (r + 31) & ~31;
  for (int c0 = 0; c0 < 2 * rp; c0 += NT / 8) {
    const int col = c0 + (int)threadIdx.x / 8, pass = col / rp, j = col % rp;
    const double* w = (pass ? R.Wf : R.We) + (size_t)j * n;
    oz_split_vec<8>([&](int l) { return w[l]; }, j < r ? n : 0, np, R.Wsl + (size_t)col * OZ_S * np, np,
                    &R.Wexp[col], true);
  }
}

// Real factors: E = A_CB W_E and F^T = A_BC^T W_F for one 64-row panel of C,
// with the panel rows and the columns of W cut into digit slices (row and
// column scales) and the slice products summed exactly on the tensor cores as
// in the Schur update; E (F^T) = W 2^(e_i + f_j - 53) from one int64 per entry.
// W is taken 32 columns at a time from its precomputed slices.  A symmetric A
// gives A_BC^T = A_CB, so the panel is cut once for both products.  The rows of
// E and F^T are then sliced for the Schur update.
constexpr int OZ_NCH = 32;

__global__ void __launch_bounds__(NT, 2) k_elim_oz(ElimArgs<double> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BoxRec<double> R = a.recs[blockIdx.y];
  if (!R.ozp) return;
  const int p0 = blockIdx.x * 64;
  if (p0 >= R.c) return;
  const LevelDev<double>& L = a.L;
  const int nmax = L.nmax, g = L.g, B = R.box, k = R.k, r = R.r, c = R.c, n = k + r;
  const int np = (n + 15) & ~15, SA = OZ_S * np + 8, rp = (r + 31) & ~31;
  const size_t nn = (size_t)nmax * nmax;
  const int* perm = a.perm_in + (size_t)a.cls_idx[blockIdx.y] * nmax;
  uint16_t* As = reinterpret_cast<uint16_t*>(smraw);   // 64 x SA: panel rows
  uint16_t* Bs = As + 64 * SA;                         // OZ_NCH x SA: columns of W
  __shared__ int rexp[64], cexp[OZ_NCH], ru[64], rpos[64];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, t4 = lane & 3;
  const int rows = min(64, c - p0);
  if (tid < 64) {
    ru[tid] = -1;
    rpos[tid] = 0;
    if (tid < rows) {
      const int cm = R.cmap[p0 + tid], s = cm >> 16;
      ru[tid] = nbr_box(B, g, s % 3 - 1, s / 3 - 1);
      rpos[tid] = cm & 0xffff;
    }
  }
  __syncthreads();
  const int m0 = (warp >> 1) * 16, n0 = (warp & 1) * 16;
  const int a_row = lane & 15, a_k = (lane >> 4) * 8;
  const int b_row = ((lane >> 4) << 3) + (lane & 7), b_k = ((lane >> 3) & 1) * 8;
  const int npass = a.sym ? 1 : 2;
  for (int pass = 0; pass < npass; ++pass) {
    {   // panel rows: A(u, B)[pos, perm[l]] (pass 0) or A(B, u)[perm[l], pos] (pass 1)
      const int row = tid >> 2, u = ru[row], pos = rpos[row];
      const double* base = nullptr;
      if (u >= 0)
        base = pass == 0 ? L.blk + ((size_t)u * 25 + off_index(u, B, g)) * nn + pos
                         : L.blk + ((size_t)B * 25 + off_index(B, u, g)) * nn + (size_t)pos * nmax;
      const size_t ls = pass == 0 ? (size_t)nmax : 1;
      oz_split_vec<4>([&](int l) { return base[(size_t)perm[l] * ls]; }, u >= 0 ? n : 0, np, As + row * SA, np,
                      &rexp[row], true);
    }
    // columns of [W_E W_F] (symmetric A) or of the pass's W
    const int c_lo = a.sym ? 0 : pass * rp, c_hi = a.sym ? 2 * rp : (pass + 1) * rp;
    for (int cc = c_lo; cc < c_hi; cc += OZ_NCH) {
      const int j0 = cc % rp;
      if (j0 >= r) continue;   // padding columns only
      __syncthreads();
      {   // one (column, slice) row of the chunk's W slices per thread
        const int col = tid >> 3, sl = tid & 7;
        const uint16_t* src = R.Wsl + (size_t)(cc + col) * OZ_S * np + (size_t)sl * np;
        uint16_t* dst = Bs + col * SA + sl * np;
        for (int q = 0; q < np; q += 8) cp_async16(dst + q, src + q);
      }
      if (tid < OZ_NCH) cexp[tid] = R.Wexp[cc + tid];
      cp_async_wait_all();
      __syncthreads();
      // all eight group sums in FP32 over the whole K (K <= 128: exact), B slices
      // loaded four at a time with the A slices that pair with them
      float acc[OZ_S][2][4];
#pragma unroll
      for (int u = 0; u < OZ_S; ++u)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[u][ni][e] = 0.f;
      for (int kk = 0; kk < np; kk += 16) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t bq[4][4];
#pragma unroll
          for (int q = 0; q < 4; ++q) ldsm_x4(bq[q], Bs + (4 * h + q) * np + (n0 + b_row) * SA + kk + b_k);
#pragma unroll
          for (int p = 0; p + 4 * h < OZ_S; ++p) {
            uint32_t af[4];
            ldsm_x4(af, As + p * np + (m0 + a_row) * SA + kk + a_k);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (p + 4 * h + q < OZ_S) {
                mma_bf16(acc[p + 4 * h + q][0], af, bq[q]);
                mma_bf16(acc[p + 4 * h + q][1], af, bq[q] + 2);
              }
          }
        }
      }
      // W = sum_u G_u 2^(39-7u), groups u and u + 1 as (G_u 2^7 + G_{u+1}) 2^(32-7u)
      long long W[2][4];
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          long long w = 0;
#pragma unroll
          for (int u = 0; u < OZ_S; u += 2) {
            const long long gv = (long long)(oz_fint(acc[u][ni][e]) * 128 + oz_fint(acc[u + 1][ni][e]));
            const int sh = 32 - OZ_BITS * u;
            w += sh >= 0 ? (gv << sh) : ((gv + (1LL << (-sh - 1))) >> (-sh));
          }
          W[ni][e] = w;
        }
      double* out = cc < rp ? R.E : R.Ft;
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int row = m0 + gq + (e >= 2 ? 8 : 0);
          const int col = n0 + ni * 8 + 2 * t4 + (e & 1), j = j0 + col;
          if (row < rows && j < r)
            out[(size_t)(p0 + row) + (size_t)j * c] = oz_ldexp_int(W[ni][e], rexp[row] + cexp[col] - 53);
        }
    }
    __syncthreads();
  }
  if (R.Esl != nullptr) {   // digit slices of this panel's rows of E and F^T for the Schur update
    const int row = tid >> 2;
    const bool act = row < rows;
    for (int q = 0; q < 2; ++q) {
      const double* src = (q == 0 ? R.E : R.Ft) + (size_t)(p0 + row);
      uint16_t* dst = (q == 0 ? R.Esl : R.Fsl) + (size_t)(p0 + (act ? row : 0)) * OZ_S * R.kp;
      int* ex = (q == 0 ? R.Eexp : R.Fexp) + p0 + (act ? row : 0);
      oz_split_vec<4>([&](int l) { return src[(size_t)l * c]; }, act ? r : 0, R.kp, dst, R.kp, ex, act);
    }
  }
}

// ------------------------------------------------------------------ complex E and F on the tensor cores


// Complex factors: E = A_CB W_E and F^T = A_BC^T W_F for one 64-row panel of C
// (any n_B: K is taken in chunks), then the rows' digit slices for the Schur
// update.
__global__ void __launch_bounds__(NT, 2) k_elim_ozc(ElimArgs<zd> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BoxRec<zd> R = a.recs[blockIdx.y];
  if (!R.ozp) return;
  const int p0 = blockIdx.x * ZCM;
  if (p0 >= R.c) return;
  const LevelDev<zd>& L = a.L;
  const int nmax = L.nmax, g = L.g, B = R.box, k = R.k, r = R.r, c = R.c, n = k + r;
  const size_t nn = (size_t)nmax * nmax;
  const int* perm = a.perm_in + (size_t)a.cls_idx[blockIdx.y] * nmax;
  uint16_t* As = reinterpret_cast<uint16_t*>(smraw);
  uint16_t* Bs = As + ZCM * ZSA;
  __shared__ int rexp[ZCM], cexp[ZCN], ru[ZCM], rpos[ZCM], sperm[256];
  const int tid = threadIdx.x, rows = min(ZCM, c - p0);
  if (tid < ZCM) {
    ru[tid] = -1;
    rpos[tid] = 0;
    if (tid < rows) {
      const int cm = R.cmap[p0 + tid], s = cm >> 16;
      ru[tid] = nbr_box(B, g, s % 3 - 1, s / 3 - 1);
      rpos[tid] = cm & 0xffff;
    }
  }
  const bool pin = n <= 256;
  if (pin)
    for (int i = tid; i < n; i += blockDim.x) sperm[i] = perm[i];
  __syncthreads();
  auto pm = [&](int l) { return pin ? sperm[l] : perm[l]; };
  for (int pass = 0; pass < 2; ++pass) {
    const zd* __restrict__ Wm = pass == 0 ? R.We : R.Wf;
    zd* out = pass == 0 ? R.E : R.Ft;
    for (int jc = 0; jc < r; jc += ZCN) {
      auto aval = [&](int i, int l) -> zd {
        const int u = ru[i], pos = rpos[i];
        return pass == 0 ? L.blk[((size_t)u * 25 + off_index(u, B, g)) * nn + (size_t)pm(l) * nmax + pos]
                         : L.blk[((size_t)B * 25 + off_index(B, u, g)) * nn + (size_t)pos * nmax + pm(l)];
      };
      auto bval = [&](int l, int q) -> zd {
        const int j = jc + q;
        return j < r ? Wm[(size_t)l + (size_t)j * n] : zd{0.0, 0.0};
      };
      tc_gemm_c(rows, n, aval, bval,
                [&](int i, int q, zd v) {
                  const int j = jc + q;
                  if (j < r) out[(size_t)(p0 + i) + (size_t)j * c] = v;
                },
                As, Bs, rexp, cexp);
    }
    if (R.Esl != nullptr) {   // digit slices of this panel's rows for the Schur update
      for (int e = tid; e < rows; e += blockDim.x)
        oz_split_row(out + p0 + e, c, r, R.kp, (pass == 0 ? R.Esl : R.Fsl) + (size_t)(p0 + e) * 2 * OZ_S * R.kp,
                     (pass == 0 ? R.Eexp : R.Fexp) + p0 + e);
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ Schur update A_CC -= E F
template <typename T> __global__ void __launch_bounds__(NT) k_schur(LevelDev<T> L, const BoxRec<T>* recs) {
  constexpr int TM = 64, KC = 16;
  const BoxRec<T> R = recs[blockIdx.y];
  const int c = R.c, r = R.r, nt = (c + TM - 1) / TM;
  if ((int)blockIdx.x >= nt * nt) return;
  const int i0 = (blockIdx.x % nt) * TM, j0 = (blockIdx.x / nt) * TM;
  const int nmax = L.nmax, g = L.g;
  const long long nn = (long long)nmax * nmax;
  __shared__ T Es[KC][TM], Fs[KC][TM];
  __shared__ long long rowb[TM], colb[TM];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  if (tid < TM) {
    const int i = i0 + tid;
    if (i < c) {
      const int cm = R.cmap[i], s = cm >> 16, pos = cm & 0xffff;
      const int u = nbr_box(R.box, g, s % 3 - 1, s / 3 - 1);
      rowb[tid] = (long long)u * 25 * nn + pos - (long long)((s / 3) * 5 + s % 3) * nn;
    }
  } else if (tid < 2 * TM) {
    const int j = j0 + tid - TM;
    if (j < c) {
      const int cm = R.cmap[j], s = cm >> 16, pos = cm & 0xffff;
      colb[tid - TM] = (long long)((s / 3) * 5 + s % 3 + 12) * nn + (long long)pos * nmax;
    }
  }
  T acc[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int w = 0; w < 4; ++w) acc[q][w] = zero<T>();
  for (int l0 = 0; l0 < r; l0 += KC) {
    __syncthreads();
    for (int e = tid; e < KC * TM; e += NT) {
      const int ii = e % TM, ll = e / TM, l = l0 + ll;
      Es[ll][ii] = (i0 + ii < c && l < r) ? R.E[i0 + ii + (size_t)l * c] : zero<T>();
      Fs[ll][ii] = (j0 + ii < c && l < r) ? R.Ft[j0 + ii + (size_t)l * c] : zero<T>();
    }
    __syncthreads();
#pragma unroll 4
    for (int ll = 0; ll < KC; ++ll) {
      T av[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { av[q] = Es[ll][tx + 16 * q]; bv[q] = Fs[ll][ty + 16 * q]; }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[q][w] = mad(acc[q][w], av[q], bv[w]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int i = i0 + tx + 16 * q, j = j0 + ty + 16 * w;
      if (i < c && j < c) {
        T* p = L.blk + rowb[tx + 16 * q] + colb[ty + 16 * w];
        *p = *p - acc[q][w];
      }
    }
}

// ------------------------------------------------------------------ Schur update on tensor cores
// A_CC -= E F for real factors with E and F^T split into OZ_S digit slices.
// (E F)_ij = 2^(e_i + f_j) sum_u 2^(-7(u+2)) G_u with G_u = sum_{p+q=u} D_p D'_q^T:
// each G_u is a sum of integer products below 2^24, so bf16 MMAs with FP32
// accumulation compute it exactly; groups u <= OZ_S-1 are kept (the rest lie
// below 2^-56 of the row/column scale, the order of an FP64 product's rounding).
// The groups are gathered in one int64 W = sum_u G_u 2^(39-7u) (the last two by
// rounding right shifts, an error below 2^-53 of the scale), so
// (E F)_ij = W 2^(e_i + f_j - 53): one conversion and one scaling per entry.
// 64 x 32 tile per CTA, 8 warps of 16 x 16.  All eight group sums of a warp's
// tile stay in FP32 registers over the whole K: each is an integer below
// 10 2^12 K, exact for K <= 384, so the groups are combined into W once per
// tile (and once per 384 entries of K beyond that) instead of once per chunk.
// Per K step of 16 the B fragments are loaded once, four slices at a time, and
// the A slices that pair with them, for the 36 products p + q <= 7.  K is staged in chunks of
// 32, double-buffered with cp.async.
constexpr int SRK = 32, SRSA = OZ_S * SRK + 8;   // real Schur: K chunk and slice-row stride
constexpr int SR_M = 64, SR_N = 32;              // CTA tile
constexpr int SR_BUF = (SR_M + SR_N) * SRSA;     // one stage of slices (uint16)
constexpr int SR_FLUSH = 12;                     // chunks between int64 gathers (12 x 32 = 384)

__global__ void __launch_bounds__(NT, 2) k_schur_oz(LevelDev<double> L, const BoxRec<double>* recs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BoxRec<double> R = recs[blockIdx.y];
  const int c = R.c, kp = R.kp, ntr = (c + SR_M - 1) / SR_M, ntc = (c + SR_N - 1) / SR_N;
  if ((int)blockIdx.x >= ntr * ntc) return;
  const int i0 = (blockIdx.x % ntr) * SR_M, j0 = (blockIdx.x / ntr) * SR_N;
  const int SA = SRSA;
  uint16_t* stage = reinterpret_cast<uint16_t*>(smraw);   // two stages: A rows then B rows
  __shared__ long long rowb[SR_M], colb[SR_N];
  __shared__ int rexp[SR_M], cexp[SR_N];
  const int nmax = L.nmax, g = L.g;
  const long long nn = (long long)nmax * nmax;
  const int tid = threadIdx.x;
  if (tid < SR_M) {
    const int i = i0 + tid;
    if (i < c) {
      const int cm = R.cmap[i], s = cm >> 16, pos = cm & 0xffff;
      const int u = nbr_box(R.box, g, s % 3 - 1, s / 3 - 1);
      rowb[tid] = (long long)u * 25 * nn + pos - (long long)((s / 3) * 5 + s % 3) * nn;
      rexp[tid] = R.Eexp[i];
    }
  } else if (tid < SR_M + SR_N) {
    const int j = j0 + tid - SR_M;
    if (j < c) {
      const int cm = R.cmap[j], s = cm >> 16, pos = cm & 0xffff;
      colb[tid - SR_M] = (long long)((s / 3) * 5 + s % 3 + 12) * nn + (long long)pos * nmax;
      cexp[tid - SR_M] = R.Fexp[j];
    }
  }
  const int warp = tid >> 5, lane = tid & 31, gq = lane >> 2, t4 = lane & 3;
  const int m0 = (warp >> 1) * 16, n0 = (warp & 1) * 16;
  const int a_row = lane & 15, a_k = (lane >> 4) * 8;
  const int b_row = ((lane >> 4) << 3) + (lane & 7), b_k = ((lane >> 3) & 1) * 8;
  // slices of rows i0.. of E and j0.. of F^T, entries kc .. kc + kl of K
  auto load = [&](int buf, int kc) {
    const int kl = min(SRK, kp - kc), cpr = OZ_S * (kl / 8);   // 16-byte chunks per row
    uint16_t* As = stage + buf * SR_BUF;
    for (int e = tid; e < (SR_M + SR_N) * cpr; e += NT) {
      const int row = e / cpr, rem = e % cpr, sl = rem / (kl / 8), ch = rem % (kl / 8);
      const bool isA = row < SR_M;
      const int gi = isA ? i0 + row : j0 + row - SR_M;
      uint16_t* d = As + row * SA + sl * SRK + ch * 8;
      if (gi < c)
        cp_async16(d, (isA ? R.Esl : R.Fsl) + (size_t)gi * OZ_S * kp + (size_t)sl * kp + kc + ch * 8);
      else
        *reinterpret_cast<uint4*>(d) = make_uint4(0, 0, 0, 0);
    }
    cp_async_commit();
  };
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
  // W += sum_u G_u 2^(39-7u), groups u and u + 1 as (G_u 2^7 + G_{u+1}) 2^(32-7u)
  // (exact in int32: |G| < 2^23); then the FP32 sums restart from zero
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
  const int nch = (kp + SRK - 1) / SRK;
  // the tile of A_CC, prefetched into the idle stage while the last chunk is multiplied
  double* Cs = reinterpret_cast<double*>(stage + (nch & 1) * SR_BUF);   // SR_M x SR_N, ld SR_M
  load(0, 0);
  for (int ci = 0; ci < nch; ++ci) {
    if (ci + 1 < nch) {
      load((ci + 1) & 1, (ci + 1) * SRK);
    } else {
      if (ci == 0) __syncthreads();   // rowb and colb
      for (int e = tid; e < SR_M * SR_N; e += NT) {
        const int row = e % SR_M, col = e / SR_M;
        if (i0 + row < c && j0 + col < c) cp_async8(Cs + e, L.blk + rowb[row] + colb[col]);
      }
      cp_async_commit();
    }
    cp_async_wait_group<1>();
    __syncthreads();
    const uint16_t* As = stage + (ci & 1) * SR_BUF;
    const uint16_t* Bs = As + SR_M * SA;
    const int kl = min(SRK, kp - ci * SRK);
    for (int kk = 0; kk < kl; kk += 16) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {   // slices q = 4h .. 4h + 3 of B, then every A slice p <= 7 - q
        uint32_t bq[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) ldsm_x4(bq[q], Bs + (n0 + b_row) * SA + (4 * h + q) * SRK + kk + b_k);
#pragma unroll
        for (int p = 0; p + 4 * h < OZ_S; ++p) {
          uint32_t af[4];
          ldsm_x4(af, As + (m0 + a_row) * SA + p * SRK + kk + a_k);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (p + 4 * h + q < OZ_S) {
              mma_bf16(acc[p + 4 * h + q][0], af, bq[q]);
              mma_bf16(acc[p + 4 * h + q][1], af, bq[q] + 2);
            }
        }
      }
    }
    if ((ci + 1) % SR_FLUSH == 0 && ci + 1 < nch) gather();
    __syncthreads();   // the stage read here is refilled by the next iteration's load
  }
  gather();
  cp_async_wait_group<0>();
  __syncthreads();
#pragma unroll
  for (int ni = 0; ni < 2; ++ni)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int row = m0 + gq + (e >= 2 ? 8 : 0);
      const int col = n0 + ni * 8 + 2 * t4 + (e & 1);
      if (i0 + row < c && j0 + col < c) {
        const double v = oz_ldexp_int(W[ni][e], rexp[row] + cexp[col] - 53);
        L.blk[rowb[row] + colb[col]] = Cs[row + col * SR_M] - v;
      }
    }
}

// The same update on the 5th-generation tensor cores (tcgen05): one thread
// issues the slice products into tensor memory.  A CTA of 256 threads owns 128
// rows (of E) x 32 columns (rows of F^T) of A_CC; group sum G_u (u = p + q)
// accumulates in TMEM columns 32u .. 32u + 31 (256 columns, two CTAs per SM) in
// FP32 over the whole K (exact for kp <= 384, checked by the host); per K step
// of 16 it takes eight products, A slice p against the stacked B slices
// 0 .. 7 - p (N = 32 (8 - p)).  K is staged
// in chunks of 32 in the no-swizzle K-major layout of 8-row x 16-byte core
// matrices: slice p, row m, entries 8g .. 8g + 7 of the chunk at
// p * rows * 64 + ((m / 8) * 4 + g) * 128 + (m % 8) * 16 bytes (LBO 128, SBO 512).
// After the last chunk every thread reads the eight groups of 16 columns of its
// row (warps w and w + 4 share TMEM lanes 32 (w % 4) ..) with
// tcgen05.ld, gathers each entry into one int64 as k_schur_oz does (same integer
// arithmetic, same result) and subtracts it from the entries of A_CC, which it
// loaded while the last products ran.  A barrier wait that runs out (after
// `polls` polls) sets RSS_ETIMEOUT in *err; the CTA then waits, with the much
// longer limit ST_DRAIN_POLLS, for the products it already issued to finish
// (they write its tensor memory), frees its tensor memory and returns.
constexpr int ST_M = 128, ST_N = 32, ST_KC = 32, ST_NT = 256;
constexpr int ST_A = OZ_S * ST_M * ST_KC * 2;   // bytes of one chunk of A slices (64 KB)
constexpr int ST_B = OZ_S * ST_N * ST_KC * 2;   // 16 KB
constexpr uint32_t ST_TMEM_COLS = OZ_S * ST_N;  // 256
constexpr long long ST_POLLS = 1LL << 22;
constexpr long long ST_DRAIN_POLLS = 1LL << 26;

__global__ void __launch_bounds__(ST_NT, 2) k_schur_tc(LevelDev<double> L, const BoxRec<double>* recs, int* err,
                                                        long long polls) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_tmem;
  __shared__ long long colb[ST_N];
  __shared__ int cexp[ST_N];
  const BoxRec<double> R = recs[blockIdx.y];
  const int c = R.c, kp = R.kp, ntr = (c + ST_M - 1) / ST_M, ntc = (c + ST_N - 1) / ST_N;
  if ((int)blockIdx.x >= ntr * ntc) return;
  const int i0 = (blockIdx.x % ntr) * ST_M, j0 = (blockIdx.x / ntr) * ST_N;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, half = warp >> 2;   // TMEM lanes 32 quarter .., columns 16 half ..
  unsigned char* As = smraw;
  unsigned char* Bs = smraw + ST_A;
  const int nmax = L.nmax, g = L.g;
  const long long nn = (long long)nmax * nmax;
  const int i = i0 + 32 * quarter + lane;   // this thread's row of the tile (TMEM lane)
  long long rowb = 0;
  int rexp = 0;
  if (i < c) {
    const int cm = R.cmap[i], s = cm >> 16, pos = cm & 0xffff;
    const int u = nbr_box(R.box, g, s % 3 - 1, s / 3 - 1);
    rowb = (long long)u * 25 * nn + pos - (long long)((s / 3) * 5 + s % 3) * nn;
    rexp = R.Eexp[i];
  }
  if (tid < ST_N) {
    const int j = j0 + tid;
    colb[tid] = 0;
    cexp[tid] = 0;
    if (j < c) {
      const int cm = R.cmap[j], s = cm >> 16, pos = cm & 0xffff;
      colb[tid] = (long long)((s / 3) * 5 + s % 3 + 12) * nn + (long long)pos * nmax;
      cexp[tid] = R.Fexp[j];
    }
  }
  if (tid == 0) mbar_init(&mbar, 1);
  if (warp == 0) tmem_alloc(&s_tmem, ST_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const int nch = (kp + ST_KC - 1) / ST_KC;
  constexpr int CH = ST_N / 2;   // columns of the tile per thread
  double cv[CH];
#pragma unroll
  for (int j = 0; j < CH; ++j) cv[j] = 0.0;
  int ok = 1;
  uint32_t parity = 0;   // phase of the barrier for the chunk in flight
  for (int ci = 0; ci < nch && ok; ++ci) {
    parity = ci & 1;
    const int kc = ci * ST_KC, kl = min(ST_KC, kp - kc), ng = kl / 8;   // 16-byte pieces per slice row
    const int lg = ng == 4 ? 2 : 1;                                        // kl is 16 or 32
    for (int e = tid; e < (ST_M + ST_N) * OZ_S * ng; e += ST_NT) {
      const int row = e >> (3 + lg), rem = e & (OZ_S * ng - 1), p = rem >> lg, gg = rem & (ng - 1);
      const bool isA = row < ST_M;
      const int rr = isA ? row : row - ST_M, gi = (isA ? i0 : j0) + rr;
      unsigned char* d = (isA ? As + p * (ST_M * ST_KC * 2) : Bs + p * (ST_N * ST_KC * 2)) +
                         ((rr / 8) * 4 + gg) * 128 + (rr % 8) * 16;
      if (gi < c)
        cp_async16(d, (isA ? R.Esl : R.Fsl) + (size_t)gi * OZ_S * kp + (size_t)p * kp + kc + gg * 8);
      else
        *reinterpret_cast<uint4*>(d) = make_uint4(0, 0, 0, 0);
    }
    if (ci + 1 == nch && i < c) {   // the entries of A_CC this thread updates, loaded under the last products
#pragma unroll
      for (int j = 0; j < CH; ++j)
        if (j0 + CH * half + j < c) cv[j] = L.blk[rowb + colb[CH * half + j]];
    }
    cp_async_wait_all();
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      // the B slices are stacked along N (slice q = rows 32q .. 32q + 31, SBO 512
      // throughout), so one product of A slice p with slices 0 .. 7 - p written at
      // TMEM column 32p puts A_p B_q^T into the columns of group p + q
      tc_fence_after();
      for (int s = 0; s < kl / 16; ++s) {
        const uint64_t bd = umma_desc(smem_u32(Bs + s * 256), 128, 512);
#pragma unroll
        for (int p = 0; p < OZ_S; ++p) {
          const uint64_t ad = umma_desc(smem_u32(As + p * (ST_M * ST_KC * 2) + s * 256), 128, 512);
          umma_bf16(tmem + ST_N * p, ad, bd, umma_idesc_bf16(ST_M, ST_N * (OZ_S - p)),
                    (ci > 0 || s > 0 || p > 0) ? 1u : 0u);
        }
      }
      umma_commit(&mbar);
    }
    // one warp polls the barrier; the others wait at the block barrier without issuing
    int got = 1;
    if (warp == 0) got = mbar_wait(&mbar, parity, polls) ? 1 : 0;
    ok = __syncthreads_and(got);
  }
  tc_fence_after();
  if (ok) {
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16) + CH * half;
#pragma unroll
    for (int c0 = 0; c0 < CH; c0 += 8) {
      uint32_t gr[OZ_S][8];
#pragma unroll
      for (int u = 0; u < OZ_S; ++u) tmem_ld8(gr[u], lane_base + ST_N * u + c0);
      tmem_ld_wait();
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        long long w = 0;
#pragma unroll
        for (int u = 0; u < OZ_S; u += 2) {
          const long long gv = (long long)(oz_fint(__uint_as_float(gr[u][jj])) * 128 +
                                           oz_fint(__uint_as_float(gr[u + 1][jj])));
          const int sh = 32 - OZ_BITS * u;
          w += sh >= 0 ? (gv << sh) : ((gv + (1LL << (-sh - 1))) >> (-sh));
        }
        const int j = CH * half + c0 + jj;
        if (i < c && j0 + j < c) L.blk[rowb + colb[j]] = cv[c0 + jj] - oz_ldexp_int(w, rexp + cexp[j] - 53);
      }
    }
  } else {
    if (tid == 0) atomicExch(err, (int)RSS_ETIMEOUT);
    if (warp == 0) mbar_wait(&mbar, parity, ST_DRAIN_POLLS);   // products in flight finish before the TMEM is freed
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, ST_TMEM_COLS);
}

// The same update with one CTA per 128-row block of A_CC that walks the
// 32-column tiles of its rows (kp <= 64): the A slices of the block are staged
// once and stay in shared memory, and the group sums alternate between two
// 256-column halves of tensor memory, so the gathering and read-modify-write of
// tile t - 1 run while the products of tile t are in flight.  The B slices of
// tile t + 1 are staged while tile t - 1 is gathered (its products, the last
// reader of that buffer, are done), and the entries of A_CC of a tile are
// loaded one tile ahead.  Every warp polls the products' barrier itself; one
// block barrier ends each step.  Per tile the same slice products, the same
// exact FP32 group sums and the same integer gathering as k_schur_tc: the same
// bits.  A barrier wait that runs out sets RSS_ETIMEOUT; the CTA then drains
// the products it issued (up to two tiles, the long limit), frees its tensor
// memory and returns.
constexpr int SRW_KP = 64;                  // largest kp of the row-block form
constexpr uint32_t SRW_TMEM_COLS = 2 * ST_TMEM_COLS;
constexpr int SRW_NT = 512;   // four warps per 32 TMEM lanes, 8 columns of a tile per thread

__global__ void __launch_bounds__(SRW_NT, 1) k_schur_tc_rows(LevelDev<double> L, const BoxRec<double>* recs, int* err,
                                                             long long polls) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ long long colb[3][ST_N];   // column data of tile t in buffer t % 3
  __shared__ int cexp[3][ST_N];
  const BoxRec<double> R = recs[blockIdx.y];
  const int c = R.c, kp = R.kp, ntr = (c + ST_M - 1) / ST_M, ntc = (c + ST_N - 1) / ST_N;
  if ((int)blockIdx.x >= ntr) return;
  const int i0 = blockIdx.x * ST_M;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, half = warp >> 2;   // TMEM lanes 32 quarter .., columns CH half ..
  const int nch = (kp + ST_KC - 1) / ST_KC;   // 1 or 2
  unsigned char* As = smraw;                   // nch chunks of ST_A
  unsigned char* Bs = smraw + nch * ST_A;      // two buffers of nch chunks of ST_B
  const int nmax = L.nmax, g = L.g;
  const long long nn = (long long)nmax * nmax;
  const int i = i0 + 32 * quarter + lane;
  long long rowb = 0;
  int rexp = 0;
  if (i < c) {
    const int cm = R.cmap[i], s = cm >> 16, pos = cm & 0xffff;
    const int u = nbr_box(R.box, g, s % 3 - 1, s / 3 - 1);
    rowb = (long long)u * 25 * nn + pos - (long long)((s / 3) * 5 + s % 3) * nn;
    rexp = R.Eexp[i];
  }
  // stage the B slices of tile t into buffer t & 1 and its column data into buffer t % 3
  auto stage_b = [&](int t) {
    const int j0 = t * ST_N;
    unsigned char* Bb = Bs + (t & 1) * nch * ST_B;
    for (int ci = 0; ci < nch; ++ci) {
      const int kc = ci * ST_KC, kl = min(ST_KC, kp - kc), ng = kl / 8, lg = ng == 4 ? 2 : 1;
      for (int e = tid; e < ST_N * OZ_S * ng; e += SRW_NT) {
        const int rr = e >> (3 + lg), rem = e & (OZ_S * ng - 1), p = rem >> lg, gg = rem & (ng - 1);
        unsigned char* d = Bb + ci * ST_B + p * (ST_N * ST_KC * 2) + ((rr / 8) * 4 + gg) * 128 + (rr % 8) * 16;
        if (j0 + rr < c)
          cp_async16(d, R.Fsl + (size_t)(j0 + rr) * OZ_S * kp + (size_t)p * kp + kc + gg * 8);
        else
          *reinterpret_cast<uint4*>(d) = make_uint4(0, 0, 0, 0);
      }
    }
    if (tid < ST_N) {
      const int j = j0 + tid;
      long long cb = 0;
      int ce = 0;
      if (j < c) {
        const int cm = R.cmap[j], s = cm >> 16, pos = cm & 0xffff;
        cb = (long long)((s / 3) * 5 + s % 3 + 12) * nn + (long long)pos * nmax;
        ce = R.Fexp[j];
      }
      colb[t % 3][tid] = cb;
      cexp[t % 3][tid] = ce;
    }
  };
  // A slices of the row block, all chunks
  for (int ci = 0; ci < nch; ++ci) {
    const int kc = ci * ST_KC, kl = min(ST_KC, kp - kc), ng = kl / 8, lg = ng == 4 ? 2 : 1;
    for (int e = tid; e < ST_M * OZ_S * ng; e += SRW_NT) {
      const int rr = e >> (3 + lg), rem = e & (OZ_S * ng - 1), p = rem >> lg, gg = rem & (ng - 1);
      unsigned char* d = As + ci * ST_A + p * (ST_M * ST_KC * 2) + ((rr / 8) * 4 + gg) * 128 + (rr % 8) * 16;
      if (i0 + rr < c)
        cp_async16(d, R.Esl + (size_t)(i0 + rr) * OZ_S * kp + (size_t)p * kp + kc + gg * 8);
      else
        *reinterpret_cast<uint4*>(d) = make_uint4(0, 0, 0, 0);
    }
  }
  stage_b(0);
  if (ntc > 1) stage_b(1);
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
  }
  if (warp == 0) tmem_alloc(&s_tmem, SRW_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  constexpr int CH = ST_N / (SRW_NT / 128);
  double cv[CH], cvn[CH];
#pragma unroll
  for (int j = 0; j < CH; ++j) cv[j] = cvn[j] = 0.0;
  int ok = 1, failed_at = -1;
  for (int t = 0; t <= ntc && ok; ++t) {
    if (t == 0) {
      cp_async_wait_all();
      fence_async_smem();
      __syncthreads();   // A slices and the B slices of tiles 0 and 1 staged
    }
    // from tile 1 on, the barrier at the end of the previous step stands here:
    // the B slices of tile t staged, tensor memory half t & 1 drained (tile t - 2)
    if (t < ntc) {
      if (tid == 0) {
        tc_fence_after();
        const unsigned char* Bb = Bs + (t & 1) * nch * ST_B;
        const uint32_t dcol = tmem + (uint32_t)(t & 1) * ST_TMEM_COLS;
        for (int ci = 0; ci < nch; ++ci) {
          const int kl = min(ST_KC, kp - ci * ST_KC);
          for (int s = 0; s < kl / 16; ++s) {
            const uint64_t bd = umma_desc(smem_u32(Bb + ci * ST_B + s * 256), 128, 512);
#pragma unroll
            for (int p = 0; p < OZ_S; ++p) {
              const uint64_t ad = umma_desc(smem_u32(As + ci * ST_A + p * (ST_M * ST_KC * 2) + s * 256), 128, 512);
              umma_bf16(dcol + ST_N * p, ad, bd, umma_idesc_bf16(ST_M, ST_N * (OZ_S - p)),
                        (ci > 0 || s > 0 || p > 0) ? 1u : 0u);
            }
          }
        }
        umma_commit(&mbar[t & 1]);
      }
      // the entries of A_CC of tile t, read while its products run
      const int j0 = t * ST_N;
      if (i < c) {
#pragma unroll
        for (int j = 0; j < CH; ++j)
          if (j0 + CH * half + j < c) cvn[j] = L.blk[rowb + colb[t % 3][CH * half + j]];
      }
    }
    if (t >= 1) {   // tile t - 1: wait for its products, gather, update A_CC
      // every warp polls the barrier itself, so the warps that issued no products
      // start gathering while thread 0 is still issuing those of tile t
      const int tp = t - 1, b = tp & 1;
      const int got = __all_sync(0xffffffffu, mbar_wait(&mbar[b], (uint32_t)(tp >> 1) & 1u, polls) ? 1 : 0);
      if (got) {
        // the products of tile t - 1 are done, so its B buffer takes tile t + 1
        // while this tile is gathered
        if (t + 1 < ntc) stage_b(t + 1);
        tc_fence_after();
        const int j0 = tp * ST_N, cb3 = tp % 3;
        const uint32_t lane_base = tmem + (uint32_t)b * ST_TMEM_COLS + ((uint32_t)(32 * quarter) << 16) + CH * half;
#pragma unroll
        for (int c0 = 0; c0 < CH; c0 += 8) {
          uint32_t gr[OZ_S][8];
#pragma unroll
          for (int u = 0; u < OZ_S; ++u) tmem_ld8(gr[u], lane_base + ST_N * u + c0);
          tmem_ld_wait();
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            long long w = 0;
#pragma unroll
            for (int u = 0; u < OZ_S; u += 2) {
              const long long gv = (long long)(oz_fint(__uint_as_float(gr[u][jj])) * 128 +
                                               oz_fint(__uint_as_float(gr[u + 1][jj])));
              const int sh = 32 - OZ_BITS * u;
              w += sh >= 0 ? (gv << sh) : ((gv + (1LL << (-sh - 1))) >> (-sh));
            }
            const int j = CH * half + c0 + jj;
            if (i < c && j0 + j < c) L.blk[rowb + colb[cb3][j]] = cv[c0 + jj] - oz_ldexp_int(w, rexp + cexp[cb3][j] - 53);
          }
        }
      }
      cp_async_wait_all();   // the B slices of tile t + 1, for the products issued after this barrier
      fence_async_smem();
      tc_fence_before();
      // column data of tile t - 1 read; tensor memory half (t - 1) & 1 drained
      ok = __syncthreads_and(got);
      if (!ok) {
        failed_at = tp;
        break;
      }
    }
#pragma unroll
    for (int j = 0; j < CH; ++j) cv[j] = cvn[j];
  }
  if (!ok) {
    if (tid == 0) atomicExch(err, (int)RSS_ETIMEOUT);
    if (warp == 0) {   // products in flight (tiles failed_at and failed_at + 1) finish before the TMEM is freed
      mbar_wait(&mbar[failed_at & 1], (uint32_t)(failed_at >> 1) & 1u, ST_DRAIN_POLLS);
      if (failed_at + 1 < ntc)
        mbar_wait(&mbar[(failed_at + 1) & 1], (uint32_t)((failed_at + 1) >> 1) & 1u, ST_DRAIN_POLLS);
    }
  }
  cp_async_wait_all();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, SRW_TMEM_COLS);
}

// Complex factors on tcgen05: Re(E F) = Er Fr^T + Ei (-Fi)^T and
// Im(E F) = Er Fi^T + Ei Fr^T, the slices of E and F^T sharing one scale per row
// for the real and imaginary parts.  The eight Re group sums occupy TMEM columns
// 32u .. 32u + 31 and the eight Im group sums columns 256 + 32u .. (512 columns,
// one CTA per SM); per K step of 16 each A slice p (real and imaginary) takes
// four products against the stacked B slices (Fr, Fi, and -Fi, a sign-flipped
// copy made in shared memory).  A Re or Im group sum adds twice as many products
// as a real one, so it is exact in FP32 for kp <= 192 (checked by the host).  Tile,
// staging, barrier handling and gathering as in k_schur_tc.
constexpr int SZ_A = 2 * OZ_S * ST_M * ST_KC * 2;   // Er and Ei slices of one chunk (128 KB)
constexpr int SZ_B = OZ_S * ST_N * ST_KC * 2;       // one kind of B slices (16 KB): Fr, Fi, -Fi
constexpr uint32_t SZ_TMEM_COLS = 2 * OZ_S * ST_N;  // 512

__global__ void __launch_bounds__(ST_NT, 1) k_schur_tc_c(LevelDev<zd> L, const BoxRec<zd>* recs, int* err,
                                                          long long polls) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_tmem;
  __shared__ long long colb[ST_N];
  __shared__ int cexp[ST_N];
  const BoxRec<zd> R = recs[blockIdx.y];
  const int c = R.c, kp = R.kp, ntr = (c + ST_M - 1) / ST_M, ntc = (c + ST_N - 1) / ST_N;
  if ((int)blockIdx.x >= ntr * ntc) return;
  const int i0 = (blockIdx.x % ntr) * ST_M, j0 = (blockIdx.x / ntr) * ST_N;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, half = warp >> 2;   // TMEM lanes 32 quarter .., columns 16 half ..
  unsigned char* As = smraw;
  unsigned char* Br = smraw + SZ_A;
  unsigned char* Bi = Br + SZ_B;
  unsigned char* Bn = Bi + SZ_B;
  const int nmax = L.nmax, g = L.g;
  const long long nn = (long long)nmax * nmax;
  const int i = i0 + 32 * quarter + lane;
  long long rowb = 0;
  int rexp = 0;
  if (i < c) {
    const int cm = R.cmap[i], s = cm >> 16, pos = cm & 0xffff;
    const int u = nbr_box(R.box, g, s % 3 - 1, s / 3 - 1);
    rowb = (long long)u * 25 * nn + pos - (long long)((s / 3) * 5 + s % 3) * nn;
    rexp = R.Eexp[i];
  }
  if (tid < ST_N) {
    const int j = j0 + tid;
    colb[tid] = 0;
    cexp[tid] = 0;
    if (j < c) {
      const int cm = R.cmap[j], s = cm >> 16, pos = cm & 0xffff;
      colb[tid] = (long long)((s / 3) * 5 + s % 3 + 12) * nn + (long long)pos * nmax;
      cexp[tid] = R.Fexp[j];
    }
  }
  if (tid == 0) mbar_init(&mbar, 1);
  if (warp == 0) tmem_alloc(&s_tmem, SZ_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const int nch = (kp + ST_KC - 1) / ST_KC;
  constexpr int CH = ST_N / 2;
  zd cv[CH];
#pragma unroll
  for (int j = 0; j < CH; ++j) cv[j] = zd{0.0, 0.0};
  int ok = 1;
  uint32_t parity = 0;
  for (int ci = 0; ci < nch && ok; ++ci) {
    parity = ci & 1;
    const int kc = ci * ST_KC, kl = min(ST_KC, kp - kc), ng = kl / 8;
    const int lg = ng == 4 ? 2 : 1;
    // 16 slices per row (8 real, 8 imaginary): rows of E into As, rows of F^T into Br / Bi
    for (int e = tid; e < (ST_M + ST_N) * 2 * OZ_S * ng; e += ST_NT) {
      const int row = e >> (4 + lg), rem = e & (2 * OZ_S * ng - 1), sl = rem >> lg, gg = rem & (ng - 1);
      const bool isA = row < ST_M;
      const int rr = isA ? row : row - ST_M, gi = (isA ? i0 : j0) + rr;
      unsigned char* base = isA ? As + sl * (ST_M * ST_KC * 2)
                                : (sl < OZ_S ? Br + sl * (ST_N * ST_KC * 2) : Bi + (sl - OZ_S) * (ST_N * ST_KC * 2));
      unsigned char* d = base + ((rr / 8) * 4 + gg) * 128 + (rr % 8) * 16;
      if (gi < c)
        cp_async16(d, (isA ? R.Esl : R.Fsl) + (size_t)gi * 2 * OZ_S * kp + (size_t)sl * kp + kc + gg * 8);
      else
        *reinterpret_cast<uint4*>(d) = make_uint4(0, 0, 0, 0);
    }
    if (ci + 1 == nch && i < c) {
#pragma unroll
      for (int j = 0; j < CH; ++j)
        if (j0 + CH * half + j < c) cv[j] = L.blk[rowb + colb[CH * half + j]];
    }
    cp_async_wait_all();
    __syncthreads();
    for (int e = tid; e < SZ_B / 16; e += ST_NT) {   // -Fi: flip the sign bit of every bf16
      uint4 v = reinterpret_cast<const uint4*>(Bi)[e];
      v.x ^= 0x80008000u; v.y ^= 0x80008000u; v.z ^= 0x80008000u; v.w ^= 0x80008000u;
      reinterpret_cast<uint4*>(Bn)[e] = v;
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int s = 0; s < kl / 16; ++s) {
        const uint64_t br = umma_desc(smem_u32(Br + s * 256), 128, 512);
        const uint64_t bi = umma_desc(smem_u32(Bi + s * 256), 128, 512);
        const uint64_t bn = umma_desc(smem_u32(Bn + s * 256), 128, 512);
#pragma unroll
        for (int p = 0; p < OZ_S; ++p) {
          const uint64_t ar = umma_desc(smem_u32(As + p * (ST_M * ST_KC * 2) + s * 256), 128, 512);
          const uint64_t ai = umma_desc(smem_u32(As + (OZ_S + p) * (ST_M * ST_KC * 2) + s * 256), 128, 512);
          const uint32_t idesc = umma_idesc_bf16(ST_M, ST_N * (OZ_S - p));
          const uint32_t acc = (ci > 0 || s > 0 || p > 0) ? 1u : 0u;
          umma_bf16(tmem + ST_N * p, ar, br, idesc, acc);                        // Re += Er Fr^T
          umma_bf16(tmem + ST_N * p, ai, bn, idesc, 1u);                         // Re += Ei (-Fi)^T
          umma_bf16(tmem + OZ_S * ST_N + ST_N * p, ar, bi, idesc, acc);          // Im += Er Fi^T
          umma_bf16(tmem + OZ_S * ST_N + ST_N * p, ai, br, idesc, 1u);           // Im += Ei Fr^T
        }
      }
      umma_commit(&mbar);
    }
    int got = 1;
    if (warp == 0) got = mbar_wait(&mbar, parity, polls) ? 1 : 0;
    ok = __syncthreads_and(got);
  }
  tc_fence_after();
  if (ok) {
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16) + CH * half;
#pragma unroll
    for (int c0 = 0; c0 < CH; c0 += 8) {
      long long w[2][8];
#pragma unroll
      for (int part = 0; part < 2; ++part) {   // Re, then Im
        uint32_t gr[OZ_S][8];
#pragma unroll
        for (int u = 0; u < OZ_S; ++u) tmem_ld8(gr[u], lane_base + part * OZ_S * ST_N + ST_N * u + c0);
        tmem_ld_wait();
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          long long acc = 0;
#pragma unroll
          for (int u = 0; u < OZ_S; u += 2) {
            const long long gv = (long long)(oz_fint(__uint_as_float(gr[u][jj])) * 128 +
                                             oz_fint(__uint_as_float(gr[u + 1][jj])));
            const int sh = 32 - OZ_BITS * u;
            acc += sh >= 0 ? (gv << sh) : ((gv + (1LL << (-sh - 1))) >> (-sh));
          }
          w[part][jj] = acc;
        }
      }
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int j = CH * half + c0 + jj;
        if (i < c && j0 + j < c) {
          const int sx = rexp + cexp[j] - 53;
          const zd o = cv[c0 + jj];
          L.blk[rowb + colb[j]] = zd{o.x - oz_ldexp_int(w[0][jj], sx), o.y - oz_ldexp_int(w[1][jj], sx)};
        }
      }
    }
  } else {
    if (tid == 0) atomicExch(err, (int)RSS_ETIMEOUT);
    if (warp == 0) mbar_wait(&mbar, parity, ST_DRAIN_POLLS);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, SZ_TMEM_COLS);
}

// Complex factors: Re(E F) = Er Fr^T - Ei Fi^T and Im(E F) = Er Fi^T + Ei Fr^T
// (F^T rows split as Fr, Fi), each group sum exact as in the real case; the
// sign of -Ei is flipped on the bf16 fragment bits.  64 x 32 tile per CTA,
// 8 warps of 16 x 16; K (the slices' length kp) in chunks of 32.  Row and
// column scales are fixed per row, so the int64 sums of the chunks add exactly
// (|W| <= kp 2^53).
constexpr int SCK = 32, SCSA = 2 * OZ_S * SCK + 8;

__global__ void __launch_bounds__(NT) k_schur_oz_c(LevelDev<zd> L, const BoxRec<zd>* recs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BoxRec<zd> R = recs[blockIdx.y];
  const int c = R.c, kp = R.kp;
  const int ntr = (c + 63) / 64, ntc = (c + 31) / 32;
  if ((int)blockIdx.x >= ntr * ntc) return;
  const int i0 = (blockIdx.x % ntr) * 64, j0 = (blockIdx.x / ntr) * 32;
  const int SA = SCSA;                          // row: 8 real then 8 imaginary slices of one chunk
  uint16_t* As = reinterpret_cast<uint16_t*>(smraw);
  uint16_t* Bs = As + 64 * SA;
  __shared__ long long rowb[64], colb[32];
  __shared__ int rexp[64], cexp[32];
  const int nmax = L.nmax, g = L.g;
  const long long nn = (long long)nmax * nmax;
  const int tid = threadIdx.x;
  if (tid < 64) {
    const int i = i0 + tid;
    if (i < c) {
      const int cm = R.cmap[i], s = cm >> 16, pos = cm & 0xffff;
      const int u = nbr_box(R.box, g, s % 3 - 1, s / 3 - 1);
      rowb[tid] = (long long)u * 25 * nn + pos - (long long)((s / 3) * 5 + s % 3) * nn;
      rexp[tid] = R.Eexp[i];
    }
  } else if (tid < 96) {
    const int j = j0 + tid - 64;
    if (j < c) {
      const int cm = R.cmap[j], s = cm >> 16, pos = cm & 0xffff;
      colb[tid - 64] = (long long)((s / 3) * 5 + s % 3 + 12) * nn + (long long)pos * nmax;
      cexp[tid - 64] = R.Fexp[j];
    }
  }
  const int warp = tid >> 5, lane = tid & 31, gq = lane >> 2, t4 = lane & 3;
  const int m0 = (warp >> 1) * 16, n0 = (warp & 1) * 16;
  const int a_row = lane & 15, a_k = (lane >> 4) * 8;
  const int b_row = ((lane >> 4) << 3) + (lane & 7), b_k = ((lane >> 3) & 1) * 8;
  long long Wr[2][4], Wi[2][4];
#pragma unroll
  for (int ni = 0; ni < 2; ++ni)
#pragma unroll
    for (int e = 0; e < 4; ++e) { Wr[ni][e] = 0; Wi[ni][e] = 0; }
  for (int kc = 0; kc < kp; kc += SCK) {
    const int kl = min(SCK, kp - kc), cpr = 2 * OZ_S * (kl / 8);   // 16-byte chunks per row
    __syncthreads();
    for (int e = tid; e < 96 * cpr; e += NT) {
      const int row = e / cpr, rem = e % cpr, sl = rem / (kl / 8), ch = rem % (kl / 8);
      const bool isA = row < 64;
      const int rr = isA ? row : row - 64;
      uint16_t* d = (isA ? As : Bs) + rr * SA + sl * SCK + ch * 8;
      const int gi = (isA ? i0 : j0) + rr;
      if (gi < c)
        cp_async16(d, (isA ? R.Esl : R.Fsl) + (size_t)gi * 2 * OZ_S * kp + (size_t)sl * kp + kc + ch * 8);
      else
        *reinterpret_cast<uint4*>(d) = make_uint4(0, 0, 0, 0);
    }
    cp_async_wait_all();
    __syncthreads();
    // groups u and u + 1 together, combined exactly in int32 (|G| < 2^22)
#pragma unroll 1
    for (int u = 0; u < OZ_S; u += 2) {
      float cr0[2][4], ci0[2][4], cr1[2][4], ci1[2][4];
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int e = 0; e < 4; ++e) cr0[ni][e] = ci0[ni][e] = cr1[ni][e] = ci1[ni][e] = 0.f;
      for (int p = 0; p <= u + 1; ++p) {
        const uint16_t* Ar = As + p * SCK;
        const uint16_t* Ai = As + (OZ_S + p) * SCK;
        for (int kk = 0; kk < kl; kk += 16) {
          uint32_t ar[4], ai[4], ain[4], br[4], bi[4];
          ldsm_x4(ar, Ar + (m0 + a_row) * SA + kk + a_k);
          ldsm_x4(ai, Ai + (m0 + a_row) * SA + kk + a_k);
#pragma unroll
          for (int i = 0; i < 4; ++i) ain[i] = ai[i] ^ 0x80008000u;
          ldsm_x4(br, Bs + (u + 1 - p) * SCK + (n0 + b_row) * SA + kk + b_k);
          ldsm_x4(bi, Bs + (OZ_S + u + 1 - p) * SCK + (n0 + b_row) * SA + kk + b_k);
#pragma unroll
          for (int ni = 0; ni < 2; ++ni) {
            mma_bf16(cr1[ni], ar, br + 2 * ni);
            mma_bf16(cr1[ni], ain, bi + 2 * ni);
            mma_bf16(ci1[ni], ar, bi + 2 * ni);
            mma_bf16(ci1[ni], ai, br + 2 * ni);
          }
          if (p <= u) {
            ldsm_x4(br, Bs + (u - p) * SCK + (n0 + b_row) * SA + kk + b_k);
            ldsm_x4(bi, Bs + (OZ_S + u - p) * SCK + (n0 + b_row) * SA + kk + b_k);
#pragma unroll
            for (int ni = 0; ni < 2; ++ni) {
              mma_bf16(cr0[ni], ar, br + 2 * ni);
              mma_bf16(cr0[ni], ain, bi + 2 * ni);
              mma_bf16(ci0[ni], ar, bi + 2 * ni);
              mma_bf16(ci0[ni], ai, br + 2 * ni);
            }
          }
        }
      }
      const int sh = 32 - OZ_BITS * u;
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const long long gr = (long long)(oz_fint(cr0[ni][e]) * 128 + oz_fint(cr1[ni][e]));
          const long long gi = (long long)(oz_fint(ci0[ni][e]) * 128 + oz_fint(ci1[ni][e]));
          if (sh >= 0) {
            Wr[ni][e] += gr << sh;
            Wi[ni][e] += gi << sh;
          } else {
            Wr[ni][e] += (gr + (1LL << (-sh - 1))) >> (-sh);
            Wi[ni][e] += (gi + (1LL << (-sh - 1))) >> (-sh);
          }
        }
    }
  }
#pragma unroll
  for (int ni = 0; ni < 2; ++ni)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int row = m0 + gq + (e >= 2 ? 8 : 0);
      const int col = n0 + ni * 8 + 2 * t4 + (e & 1);
      if (i0 + row < c && j0 + col < c) {
        const int sx = rexp[row] + cexp[col] - 53;
        zd* ptr = L.blk + rowb[row] + colb[col];
        const zd o = *ptr;
        *ptr = zd{o.x - oz_ldexp_int(Wr[ni][e], sx), o.y - oz_ldexp_int(Wi[ni][e], sx)};
      }
    }
}

// ------------------------------------------------------------------ merge (Section 2.4)
template <typename T> __global__ void __launch_bounds__(NT) k_merge_pts(LevelDev<T> C, LevelDev<T> P) {
  const int Pb = blockIdx.x, gp = P.g, px = Pb % gp, py = Pb / gp;
  __shared__ int ch[4], off[5];
  if (threadIdx.x == 0) {
    int o = 0;
    for (int q = 0; q < 4; ++q) {
      ch[q] = (2 * py + q / 2) * C.g + 2 * px + q % 2;   // SW, SE, NW, NE
      off[q] = o;
      o += C.nact[ch[q]];
    }
    off[4] = o;
    P.n[Pb] = o;
    P.nact[Pb] = o;
  }
  __syncthreads();
  for (int q = 0; q < 4; ++q)
    for (int i = threadIdx.x; i < off[q + 1] - off[q]; i += blockDim.x)
      P.pts[Pb * P.nmax + off[q] + i] = C.pts[ch[q] * C.nmax + C.act[ch[q] * C.nmax + i]];
  for (int i = threadIdx.x; i < off[4]; i += blockDim.x) P.act[Pb * P.nmax + i] = i;
}

template <typename T>
__global__ void __launch_bounds__(NT) k_merge_blk(LevelDev<T> C, LevelDev<T> P, const int2* __restrict__ ixy,
                                                  const T* __restrict__ tab, KParams kp, int side) {
  // dynamic: the source (child slot << 16 | position in the child) and the grid
  // coordinates of every row and every column of the parent block
  extern __shared__ __align__(16) int msm[];
  const int u = blockIdx.x / 25, o = blockIdx.x % 25;
  const int v = nbr_box(u, P.g, o % 5 - 2, o / 5 - 2);
  if (v < 0) return;
  __shared__ int cu[4], cv[4], ou[5], ov[5];
  __shared__ long long pbase[16];   // child pair (qa, qb): start of its stored block, or -1 (never stored)
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
    for (int q = 0; q < 4; ++q) {
      cu[q] = (2 * (u / P.g) + q / 2) * C.g + 2 * (u % P.g) + q % 2;
      cv[q] = (2 * (v / P.g) + q / 2) * C.g + 2 * (v % P.g) + q % 2;
      ou[q] = a; a += C.nact[cu[q]];
      ov[q] = b; b += C.nact[cv[q]];
    }
    ou[4] = a; ov[4] = b;
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    const int a = cu[threadIdx.x >> 2], b = cv[threadIdx.x & 3];
    pbase[threadIdx.x] = cheb(a, b, C.g) <= 2 ? ((long long)a * 25 + off_index(a, b, C.g)) * C.nmax * C.nmax : -1;
  }
  const int nr = ou[4], ncl = ov[4];
  int* rsrc = msm;
  int* csrc = msm + P.nmax;
  int2* rxy = reinterpret_cast<int2*>(msm + 2 * P.nmax);
  int2* cxy = rxy + P.nmax;
  for (int ip = threadIdx.x; ip < nr; ip += blockDim.x) {
    int q = 0;
    while (ou[q + 1] <= ip) ++q;
    const int pos = C.act[cu[q] * C.nmax + ip - ou[q]];
    rsrc[ip] = (q << 16) | pos;
    rxy[ip] = ixy[C.pts[cu[q] * C.nmax + pos]];
  }
  for (int jp = threadIdx.x; jp < ncl; jp += blockDim.x) {
    int q = 0;
    while (ov[q + 1] <= jp) ++q;
    const int pos = C.act[cv[q] * C.nmax + jp - ov[q]];
    csrc[jp] = (q << 16) | pos;
    cxy[jp] = ixy[C.pts[cv[q] * C.nmax + pos]];
  }
  __syncthreads();
  T* A = P.blk + ((size_t)u * 25 + o) * P.nmax * P.nmax;
  // the 4 x 4 child pairs in one pass over the parent block, rows fastest; entry
  // e = ip + jp nr stepped by the block size without a division per entry
  if (nr == 0) return;
  const int di = (int)blockDim.x % nr, dj = (int)blockDim.x / nr;
  int ip = (int)threadIdx.x % nr, jp = (int)threadIdx.x / nr;
  for (; jp < ncl; ip += di, jp += dj) {
    if (ip >= nr) {
      ip -= nr;
      ++jp;
      if (jp >= ncl) break;
    }
    const int rs = rsrc[ip], cs = csrc[jp];
    const long long base = pbase[((rs >> 16) << 2) | (cs >> 16)];
    T val;
    if (base >= 0)   // a pair the child level stored (and may have modified)
      val = C.blk[base + (long long)(cs & 0xffff) * C.nmax + (rs & 0xffff)];
    else             // never modified: kernel evaluation (Theorem 1)
      val = aval_tab<T>(kp, tab, side, rxy[ip], cxy[jp]);
    A[(size_t)jp * P.nmax + ip] = val;
  }
}

// Child level kept for the merge only: its blocks restricted to the active
// points (the merge reads nothing else), so the full blocks can be freed
// before the parent level is allocated.  out: nbox x 25 x kmax x kmax.
template <typename T>
__global__ void __launch_bounds__(NT) k_compact_blk(LevelDev<T> C, T* __restrict__ out, int* __restrict__ pts_out,
                                                    int kmax) {
  const int u = blockIdx.x / 25, o = blockIdx.x % 25;
  const int v = nbr_box(u, C.g, o % 5 - 2, o / 5 - 2);
  const int nu = C.nact[u];
  if (o == 0)
    for (int i = threadIdx.x; i < nu; i += blockDim.x) pts_out[(size_t)u * kmax + i] = C.pts[u * C.nmax + C.act[u * C.nmax + i]];
  if (v < 0) return;
  const int nv = C.nact[v];
  const T* S = C.blk + ((size_t)u * 25 + o) * C.nmax * C.nmax;
  T* D = out + ((size_t)u * 25 + o) * kmax * kmax;
  const int* au = C.act + u * C.nmax;
  const int* av = C.act + v * C.nmax;
  for (int e = threadIdx.x; e < nu * nv; e += blockDim.x) {
    const int i = e % nu, j = e / nu;
    D[(size_t)j * kmax + i] = S[(size_t)av[j] * C.nmax + au[i]];
  }
}

// Grid coordinates of every tree index (box-major, row-major inside a leaf box)
// and the grid index iy * side + ix of every user point.
__global__ void k_grid_coords(int2* ixy, int32_t* u2g, const int32_t* u2t, long long n, int gL, int ls,
                              int side) {
  const int leaf = ls * ls;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / leaf), l = (int)(t % leaf);
    ixy[t] = make_int2((b % gL) * ls + l % ls, (b / gL) * ls + l / ls);
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long t = u2t[i];
    const int b = (int)(t / leaf), l = (int)(t % leaf);
    u2g[i] = ((b / gL) * ls + l / ls) * side + (b % gL) * ls + l % ls;
  }
}

// Leaf level: box b holds tree indices b * leaf + i, all active.
__global__ void k_leaf_init(int* pts, int* act, int* n, int* nact, int nbox, int leaf) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)nbox * leaf;
       e += (long long)gridDim.x * blockDim.x) {
    pts[e] = (int)e;
    act[e] = (int)(e % leaf);
    if (e % leaf == 0) n[e / leaf] = nact[e / leaf] = leaf;
  }
}

__global__ void k_iota_rows(int* act, int nbox, int kmax) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)nbox * kmax;
       e += (long long)gridDim.x * blockDim.x)
    act[e] = (int)(e % kmax);
}

// ------------------------------------------------------------------ dense top
template <typename T>
__global__ void __launch_bounds__(NT) k_top_assemble(LevelDev<T> L, T* D, int ntop, int* top_idx, int4 offs_lo,
                                                     int offs_hi) {
  const int offs[5] = {offs_lo.x, offs_lo.y, offs_lo.z, offs_lo.w, offs_hi};
  const int u = blockIdx.x / L.nbox, v = blockIdx.x % L.nbox;
  const int nu = L.n[u], nv = L.n[v];
  const T* A = L.blk + ((size_t)u * 25 + off_index(u, v, L.g)) * L.nmax * L.nmax;
  for (int e = threadIdx.x; e < nu * nv; e += blockDim.x) {
    const int i = e % nu, j = e / nu;
    D[(size_t)(offs[v] + j) * ntop + offs[u] + i] = A[(size_t)j * L.nmax + i];
  }
  if (v == 0)
    for (int i = threadIdx.x; i < nu; i += blockDim.x) top_idx[offs[u] + i] = L.pts[u * L.nmax + i];
}

// Blocked right-looking LU with partial pivoting for the dense top block (the
// same pivot sequence as the unblocked algorithm): per panel of 32 columns,
// k_lu_panel factors A[jb:n, jb:jb+32] in one CTA, k_lu_swap_trsm applies the
// panel's row exchanges to the other columns and forms U12 = L11^{-1} A12, and
// k_lu_update subtracts L21 U12 from the trailing block across the GPU.
constexpr int LB = 32;

template <typename T> __global__ void __launch_bounds__(1024) k_lu_panel(T* A, int n, int jb, int* piv, int* err) {
  __shared__ double s_mx[32];
  __shared__ int s_mi[32], s_piv, s_zero;
  __shared__ __align__(16) double s_dinv[2];   // 1 / pivot, one division per step
  const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = bs >> 5;
  const int je = min(n, jb + LB);
  for (int j = jb; j < je; ++j) {
    double mx = -1.0;
    int mi = INT_MAX;
    for (int i = j + tid; i < n; i += bs) {
      const double v = abs2(A[i + (size_t)j * n]);
      if (v > mx) { mx = v; mi = i; }
    }
    for (int d = 16; d > 0; d >>= 1) {
      const double om = __shfl_xor_sync(0xffffffffu, mx, d);
      const int oi = __shfl_xor_sync(0xffffffffu, mi, d);
      if (om > mx || (om == mx && oi < mi)) { mx = om; mi = oi; }
    }
    if (lane == 0) { s_mx[warp] = mx; s_mi[warp] = mi; }
    __syncthreads();
    if (warp == 0) {
      mx = lane < nw ? s_mx[lane] : -1.0;
      mi = lane < nw ? s_mi[lane] : INT_MAX;
      for (int d = 16; d > 0; d >>= 1) {
        const double om = __shfl_xor_sync(0xffffffffu, mx, d);
        const int oi = __shfl_xor_sync(0xffffffffu, mi, d);
        if (om > mx || (om == mx && oi < mi)) { mx = om; mi = oi; }
      }
      if (lane == 0) {
        s_piv = mi;
        s_zero = !(mx > 0.0);
        if (mx > 0.0) *reinterpret_cast<T*>(s_dinv) = dv(from_re<T>(1.0), A[mi + (size_t)j * n]);
      }
    }
    __syncthreads();
    if (s_zero) {   // no exchange for the remaining steps: later launches index within 0 .. n-1
      if (tid == 0) atomicExch(err, (int)RSS_ENUMERIC);
      for (int i = j + tid; i < n; i += bs) piv[i] = i;
      return;
    }
    const int p = s_piv;
    if (p != j && tid < je - jb) {   // exchange rows j and p inside the panel
      const int col = jb + tid;
      const T t = A[j + (size_t)col * n];
      A[j + (size_t)col * n] = A[p + (size_t)col * n];
      A[p + (size_t)col * n] = t;
    }
    if (tid == 0) piv[j] = p;
    __syncthreads();
    const T d = *reinterpret_cast<const T*>(s_dinv);
    for (int i = j + 1 + tid; i < n; i += bs) A[i + (size_t)j * n] = A[i + (size_t)j * n] * d;
    __syncthreads();
    const int w = je - j - 1;
    for (long long e = tid; e < (long long)(n - j - 1) * w; e += bs) {
      const int i = j + 1 + (int)(e % (n - j - 1)), col = j + 1 + (int)(e / (n - j - 1));
      A[i + (size_t)col * n] = msb(A[i + (size_t)col * n], A[i + (size_t)j * n], A[j + (size_t)col * n]);
    }
    __syncthreads();
  }
}

// one thread per column outside the panel: row exchanges, then (right of the
// panel) U12 = L11^{-1} A12 by forward substitution
template <typename T> __global__ void k_lu_swap_trsm(T* A, int n, int jb, const int* piv) {
  const int je = min(n, jb + LB);
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n - (je - jb)) return;
  if (col >= jb) col += je - jb;
  T* a = A + (size_t)col * n;
  for (int j = jb; j < je; ++j) {
    const int p = piv[j];
    if (p != j) {
      const T t = a[j];
      a[j] = a[p];
      a[p] = t;
    }
  }
  if (col >= je)
    for (int i = jb + 1; i < je; ++i) {
      T x = a[i];
      for (int l = jb; l < i; ++l) x = msb(x, A[i + (size_t)l * n], a[l]);
      a[i] = x;
    }
}

// A22 -= L21 U12, 64 x 64 tiles
template <typename T> __global__ void __launch_bounds__(NT) k_lu_update(T* A, int n, int jb) {
  const int je = min(n, jb + LB), m = n - je;
  const int nt = (m + 63) / 64;
  const int i0 = je + (blockIdx.x % nt) * 64, j0 = je + (blockIdx.x / nt) * 64;
  constexpr int KC = 16;
  __shared__ T Ls[KC][64], Us[KC][64];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int kb = je - jb;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = zero<T>();
  for (int l0 = 0; l0 < kb; l0 += KC) {
    __syncthreads();
    for (int e = tid; e < KC * 64; e += NT) {
      const int l = l0 + e / 64, ii = e % 64;
      Ls[e / 64][ii] = (l < kb && i0 + ii < n) ? A[i0 + ii + (size_t)(jb + l) * n] : zero<T>();
      Us[e / 64][ii] = (l < kb && j0 + ii < n) ? A[jb + l + (size_t)(j0 + ii) * n] : zero<T>();
    }
    __syncthreads();
    for (int l = 0; l < KC; ++l) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) { av[a] = Ls[l][tx + 16 * a]; bv[a] = Us[l][ty + 16 * a]; }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = mad(acc[a][b], av[a], bv[b]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + tx + 16 * a, j = j0 + ty + 16 * b;
      if (i < n && j < n) A[i + (size_t)j * n] = A[i + (size_t)j * n] - acc[a][b];
    }
}

// ------------------------------------------------------------------ host helpers
template <typename T> struct HostLevel {
  LevelDev<T> d{};
  std::vector<int32_t> n, nact;
};

// Level memory is stream-ordered: freeing it needs no device synchronisation.
template <typename T> void free_level(HostLevel<T>& L, cudaStream_t st) {
  pool_free(L.d.pts, st); pool_free(L.d.n, st); pool_free(L.d.act, st); pool_free(L.d.nact, st);
  pool_free(L.d.blk, st);
  L.d = LevelDev<T>{};
}

template <typename T>
rss_status alloc_level(HostLevel<T>& L, int g, int nmax, size_t& transient, cudaStream_t st) {
  L.d = LevelDev<T>{};
  L.d.g = g;
  L.d.nbox = g * g;
  L.d.nmax = nmax;
  const size_t nb = (size_t)g * g;
  auto get = [&](auto** p, size_t bytes) { return pool_malloc(reinterpret_cast<void**>(p), bytes, st); };
  const size_t bytes = sizeof(T) * nb * 25 * (size_t)nmax * nmax;
  if (get(&L.d.pts, sizeof(int) * nb * nmax) != cudaSuccess || get(&L.d.n, sizeof(int) * nb) != cudaSuccess ||
      get(&L.d.act, sizeof(int) * nb * nmax) != cudaSuccess || get(&L.d.nact, sizeof(int) * nb) != cudaSuccess ||
      get(&L.d.blk, bytes) != cudaSuccess) {
    free_level(L, st);
    rss_set_error("rss_factor: out of device memory for the stencil blocks of the " + std::to_string(g) + " x " +
                  std::to_string(g) + " level (" + std::to_string(bytes >> 20) + " MiB, " + std::to_string(nmax) +
                  " points per box)");
    return RSS_ENOMEM;
  }
  transient += bytes;
  return RSS_OK;
}

// Frees the level it watches when the factorization returns early.
template <typename T> struct LevelGuard {
  HostLevel<T>& L;
  cudaStream_t st;
  ~LevelGuard() { free_level(L, st); }
};

// Device time of a phase: events recorded on the factor's stream around it.
struct Ev {
  cudaEvent_t a = nullptr, b = nullptr;
  Ev() { cudaEventCreate(&a); cudaEventCreate(&b); }
  ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
  void start(cudaStream_t st) { cudaEventRecord(a, st); }
  void stop(cudaStream_t st) { cudaEventRecord(b, st); }
  double ms() {   // call after the stream has been synchronised
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    return t;
  }
};

// Grow-only device buffer (freed with the factorization's host frame), in the
// order of the factor's stream: the old buffer is released after the launches
// already queued that read it.
struct GrowBuf {
  cudaStream_t st;
  void* p = nullptr;
  size_t cap = 0;
  explicit GrowBuf(cudaStream_t s) : st(s) {}
  bool ensure(size_t bytes) {
    if (bytes <= cap) return true;
    pool_free(p, st);
    p = nullptr;
    cap = 0;
    if (pool_malloc(&p, bytes, st) != cudaSuccess) return false;
    cap = bytes;
    return true;
  }
  ~GrowBuf() { pool_free(p, st); }
};

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

}  // namespace

template <typename T>
rss_status factor_impl(const rss_tree* tree, const rss_params* prm, cudaStream_t st, rss_factorization* f) {
  Timer total;
  f->n = tree->n;
  f->side = tree->side;
  f->leaf = tree->leaf;
  f->gL = tree->gL;
  f->geo = tree->geo;
  f->tree_to_user = tree->tree_to_user;
  const int P = f->params.proxy_n;
  const double ratio = f->params.proxy_radius_over_side;
  const double extent = tree->side * tree->geo.hg;
  const int64_t N = tree->n;

  f->arena.st = st;
  f->d_user_to_tree = static_cast<int32_t*>(f->arena.get(sizeof(int32_t) * N));
  if (!f->d_user_to_tree) { rss_set_error("rss_factor: device arena allocation failed"); return RSS_ENOMEM; }
  RSS_CUDA(cudaMemcpyAsync(f->d_user_to_tree, tree->user_to_tree.data(), sizeof(int32_t) * N,
                           cudaMemcpyHostToDevice, st));
  int2* d_ixy = static_cast<int2*>(f->arena.get(sizeof(int2) * N));
  int* d_err = static_cast<int*>(f->arena.get(sizeof(int)));
  f->d_user_to_grid = static_cast<int32_t*>(f->arena.get(sizeof(int32_t) * N));
  if (!d_ixy || !d_err || !f->d_user_to_grid) {
    rss_set_error("rss_factor: device arena allocation failed");
    return RSS_ENOMEM;
  }
  RSS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
  k_grid_coords<<<152 * 8, NT, 0, st>>>(d_ixy, f->d_user_to_grid, f->d_user_to_tree, N, tree->gL, tree->ls,
                                        tree->side);
  RSS_LAUNCHED();
  f->launches += 1;
  if (prm->kind == RSS_HELMHOLTZ_LS) {   // w = kappa sqrt(b) per grid point (Eq. 19)
    f->d_w = static_cast<double*>(f->arena.get(sizeof(double) * N));
    if (!f->d_w) { rss_set_error("rss_factor: device arena allocation failed"); return RSS_ENOMEM; }
    k_ls_weights<<<cdiv(N, NT), NT, 0, st>>>(f->d_w, tree->side, f->geo, f->kp.kappa, f->params.bump_cx,
                                             f->params.bump_cy, f->params.bump_a);
    RSS_LAUNCHED();
    f->kp.w = f->d_w;
    f->launches += 1;
  }
  // kernel values by displacement, for the leaf blocks and the never-modified far blocks
  const int side = tree->side;
  T* d_tab = nullptr;
  RSS_CUDA(pool_malloc(reinterpret_cast<void**>(&d_tab), sizeof(T) * (size_t)(2 * side - 1) * (2 * side - 1), st));
  struct TabFree {
    T* p;
    cudaStream_t st;
    ~TabFree() { pool_free(p, st); }
  } tab_free{d_tab, st};
  Ev span;
  span.start(st);
  k_ktab<T><<<152 * 8, NT, 0, st>>>(d_tab, side, f->kp, f->geo);
  RSS_LAUNCHED();
  f->launches += 1;

  // workspaces reused across colour classes and levels
  GrowBuf gb_cls(st), gb_k(st), gb_perm(st), gb_clsidx(st), gb_Tws(st), gb_Y(st), gb_oz(st), gb_w(st);
  // leaf level
  size_t transient = 0;
  HostLevel<T> cur;
  LevelGuard<T> cur_guard{cur, st};
  int g = tree->gL;
  {
    rss_status s = alloc_level(cur, g, tree->leaf, transient, st);
    if (s != RSS_OK) return s;
    const int nbox = g * g, leaf = tree->leaf;
    std::vector<int> hn(nbox, leaf);
    k_leaf_init<<<152 * 8, NT, 0, st>>>(cur.d.pts, cur.d.act, cur.d.n, cur.d.nact, nbox, leaf);
    RSS_LAUNCHED();
    f->launches += 1;
    cur.n = hn;
    cur.nact = hn;
    Timer tg;
    Ev ev;
    ev.start(st);
    k_gen_blocks<T><<<nbox * 25, NT, 0, st>>>(cur.d, d_ixy, d_tab, f->kp, side);
    RSS_LAUNCHED();
    ev.stop(st);
    RSS_CUDA(cudaStreamSynchronize(st));
    f->t_gen += tg.ms();
    f->g_gen += ev.ms();
    f->launches += 1;
  }

  // A real symmetric kernel (Laplace, real diagonal) keeps A symmetric through the
  // eliminations, so the conjugate half of the proxy stack repeats the first half
  // and the ID of [A_MB; K_PB] alone is the same ID.
  const int half = (prm->id_rows == 0 && prm->kind == RSS_LAPLACE && prm->diag_im == 0.0) ? 1 : 0;
  // poll limit of the first barrier wait of the tensor-core Schur updates
  const long long polls = prm->wait_polls == 0 ? ST_POLLS : prm->wait_polls < 0 ? 0 : (long long)prm->wait_polls;
  // A complex symmetric kernel (Helmholtz): the ID of the real stack
  // [Re X; Im X], X = [A_MB; K_PB], which is the ID of the full stack (T real).
  const bool split = std::is_same<T, zd>::value && prm->id_rows == 0 &&
                     (prm->kind == RSS_HELMHOLTZ || prm->kind == RSS_HELMHOLTZ_LS);
  while (g >= 4) {
    const int nbox = g * g, nmax = cur.d.nmax;
    const size_t nn = (size_t)nmax * nmax;
    const double Lbox = extent / g;
    LevelInfo info;
    info.side = g;
    info.n = cur.n;
    info.k = cur.n;
    // colour classes
    std::vector<int> cls;
    std::vector<int> coff(10, 0);
    for (int col = 0; col < 9; ++col) {
      coff[col] = (int)cls.size();
      for (int by = col / 3; by < g; by += 3)
        for (int bx = col % 3; bx < g; bx += 3) cls.push_back(by * g + bx);
    }
    coff[9] = (int)cls.size();
    if (prm->class_order != 0) {   // a seeded permutation of every class (Fisher-Yates, 64-bit LCG)
      uint64_t st64 = (uint64_t)(uint32_t)prm->class_order * 0x9E3779B97F4A7C15ull + (uint64_t)g;
      for (int col = 0; col < 9; ++col)
        for (int i = coff[col + 1] - 1; i > coff[col]; --i) {
          st64 = st64 * 6364136223846793005ull + 1442695040888963407ull;
          const int j = coff[col] + (int)((st64 >> 33) % (uint64_t)(i - coff[col] + 1));
          std::swap(cls[i], cls[j]);
        }
    }
    int maxcls = 0;
    for (int col = 0; col < 9; ++col) maxcls = std::max(maxcls, coff[col + 1] - coff[col]);
    // proxy rows from one table per level where the boxes' points outnumber the
    // table's places (the fine levels); the coarse levels evaluate them per box
    const int lsz = side / g;
    T* d_ptab = nullptr;
    if ((long long)nbox * nmax >= 2LL * lsz * lsz) {
      const size_t pb = sizeof(T) * (size_t)P * lsz * lsz;
      RSS_CUDA(pool_malloc(reinterpret_cast<void**>(&d_ptab), pb, st));
      f->peak_transient = std::max(f->peak_transient, transient + pb);
      Ev evp;
      evp.start(st);
      k_proxy_tab<T><<<std::min<long long>(cdiv((long long)P * lsz * lsz, NT), 152LL * 8), NT, 0, st>>>(
          d_ptab, lsz, P, ratio * Lbox, f->geo.hg, f->kp);
      RSS_LAUNCHED();
      evp.stop(st);
      RSS_CUDA(cudaStreamSynchronize(st));
      f->g_id += evp.ms();
      info.g_id += evp.ms();
      f->launches += 1;
    }
    struct PtabFree {
      T* p;
      cudaStream_t st;
      ~PtabFree() { pool_free(p, st); }
    } ptab_free{d_ptab, st};
    if (!gb_cls.ensure(sizeof(int) * cls.size()) || !gb_k.ensure(sizeof(int) * maxcls) ||
        !gb_perm.ensure(sizeof(int) * (size_t)maxcls * nmax) || !gb_clsidx.ensure(sizeof(int) * maxcls) ||
        !gb_Tws.ensure(sizeof(T) * (size_t)maxcls * nn)) {
      rss_set_error("rss_factor: device workspace allocation failed");
      return RSS_ENOMEM;
    }
    int* d_cls = static_cast<int*>(gb_cls.p);
    int* d_k = static_cast<int*>(gb_k.p);
    int* d_perm = static_cast<int*>(gb_perm.p);
    int* d_clsidx = static_cast<int*>(gb_clsidx.p);
    T* d_Tws = static_cast<T*>(gb_Tws.p);
    RSS_CUDA(cudaMemcpyAsync(d_cls, cls.data(), sizeof(int) * cls.size(), cudaMemcpyHostToDevice, st));
    std::vector<int> hk(maxcls);
    std::vector<std::pair<int, std::unique_ptr<Ev>>> evs;   // phase (0 id, 1 elim, 2 schur), events

    // launch segments: the nine colour classes, or (the plain per-box form, kept
    // to measure what batching gains) one box per launch in the same order
    std::vector<int> segs;
    if (prm->per_box) {
      for (int i = 0; i <= (int)cls.size(); ++i) segs.push_back(i);
    } else {
      segs = coff;
    }
    for (size_t sgi = 0; sgi + 1 < segs.size(); ++sgi) {
      const int seg0 = segs[sgi];
      const int nb = segs[sgi + 1] - seg0;
      if (nb == 0) continue;
      const int* boxes = cls.data() + seg0;
      // rows of Y per box, from the host copy of the active counts
      int mmax = 0;
      std::vector<int> mrows(nb);
      for (int q = 0; q < nb; ++q) {
        const int B = boxes[q], bx = B % g, by = B / g;
        int mh = 0;
        for (int dy = -2; dy <= 2; ++dy)
          for (int dx = -2; dx <= 2; ++dx) {
            if (std::max(std::abs(dx), std::abs(dy)) != 2) continue;
            const int x = bx + dx, y = by + dy;
            if (x < 0 || y < 0 || x >= g || y >= g) continue;
            mh += cur.nact[y * g + x];
          }
        mrows[q] = half ? mh + P : 2 * (mh + P);
        mmax = std::max(mmax, mrows[q]);
      }
      const int ldY = (mmax + 1) & ~1;
      // cluster of Q CTAs per box when the class is too small to fill the GPU
      int Q = 1;
      if (prm->id_cluster >= 0) {
        const int qcap = prm->id_cluster > 0 ? std::min(prm->id_cluster, CL_QMAX) : CL_QDEF;
        while (Q < qcap && (long long)nb * Q * 2 <= 2 * 152) Q *= 2;
        Q = std::min(Q, qcap);
      }
      Timer tid_;
      evs.emplace_back(0, std::make_unique<Ev>());
      evs.back().second->start(st);
      // TC: arithmetic of the ID (double for the complex symmetric real stack)
      auto run_id = [&](auto tag) -> rss_status {
        using TC = decltype(tag);
        const size_t slot = (2 * (size_t)ldY * nmax + 2 * nn * Q) * sizeof(TC);
        const size_t ybudget = size_t(2) << 30;
        const int cap = (int)std::max<size_t>(1, std::min<size_t>(nb, ybudget / slot));
        const int nchunks = (nb + cap - 1) / cap;
        const int chunk = (nb + nchunks - 1) / nchunks;   // balanced chunks
        if (!gb_Y.ensure(slot * chunk)) {
          rss_set_error("rss_factor: device workspace allocation failed");
          return RSS_ENOMEM;
        }
        TC* d_Y = static_cast<TC*>(gb_Y.p);
        size_t smem_id =
            sizeof(TC) * ((size_t)ldY + 2 * nmax) + (size_t)nmax * (3 * sizeof(double) + 2 * sizeof(int));
        // 512 threads per CTA when every CTA of the class gets an SM of its own
        const int ntc = (sizeof(TC) == sizeof(double) && (long long)nb * Q <= 152) ? 512 : 256;
        const int pst = ntc == 512 ? cl_part_stride<512>(nmax) : cl_part_stride<256>(nmax);
        size_t smem_cl = sizeof(TC) * ((size_t)(ldY + Q - 1) / Q + 2 * (size_t)nmax + 2 * (size_t)pst) +
                         (size_t)nmax * (3 * sizeof(double) + 2 * sizeof(int));
        // G and row k of V on chip when they fit
        const size_t gsm = 16 + sizeof(TC) * ((size_t)nmax * nmax + nmax);
        const int g_sm = (Q > 1 ? smem_cl : smem_id) + gsm <= 200 * 1024 ? 1 : 0;
        if (g_sm) {
          smem_id += gsm;
          smem_cl += gsm;
        }
        if (smem_id > 220 * 1024) {
          rss_set_error("rss_factor: proxy stack of a box too tall for the on-chip reflector buffer");
          return RSS_EINVAL;
        }
        RSS_CUDA(cudaFuncSetAttribute(k_id<TC, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_id));
        auto kcl = k_id_cl<TC, T, 256>;
        if constexpr (sizeof(TC) == sizeof(double))
          if (ntc == 512) kcl = k_id_cl<TC, T, 512>;
        if (Q > 1) {
          RSS_CUDA(cudaFuncSetAttribute(kcl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cl));
          if (Q > 8) RSS_CUDA(cudaFuncSetAttribute(kcl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        }
        f->peak_transient = std::max(f->peak_transient, transient + slot * chunk);
        for (int c0 = 0; c0 < nb; c0 += chunk) {
          IdArgs<TC, T> a;
          a.L = cur.d;
          a.boxes = d_cls + seg0;
          a.base = c0;
          a.ws = d_Y;
          a.ldY = ldY;
          a.half = half;
          a.k_out = d_k;
          a.perm_out = d_perm;
          a.T_ws = d_Tws;
          a.ixy = d_ixy;
          a.kp = f->kp;
          a.geo = f->geo;
          a.eps = f->params.eps;
          a.P = P;
          a.rho = ratio * Lbox;
          a.Lbox = Lbox;
          a.g_sm = g_sm;
          a.ptab = d_ptab;
          a.lsz = lsz;
          const int cnt = std::min(chunk, nb - c0);
          if (Q > 1) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(cnt * Q);
            cfg.blockDim = dim3(ntc);
            cfg.dynamicSmemBytes = smem_cl;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = Q;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            RSS_CUDA(cudaLaunchKernelEx(&cfg, kcl, a));
          } else {
            k_id<TC, T><<<cnt, NT_ID, smem_id, st>>>(a);
          }
          RSS_LAUNCHED();
          f->launches += 1;
          f->n_id += 1;
        }
        return RSS_OK;
      };
      {
        const rss_status s_id = split ? run_id(double{}) : run_id(T{});
        if (s_id != RSS_OK) return s_id;
      }
      evs.back().second->stop(st);
      RSS_CUDA(cudaMemcpyAsync(hk.data(), d_k, sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
      RSS_CUDA(cudaStreamSynchronize(st));
      f->t_id += tid_.ms();
      const double cf = (sizeof(T) == sizeof(double) || split) ? 1.0 : 4.0;
      for (int q = 0; q < nb; ++q) {   // k steps of Householder QR on the m x n stack
        const double m = mrows[q], n = cur.n[boxes[q]], k = hk[q];
        f->f_id += cf * (4.0 * m * n * k - 2.0 * k * k * (m + n) + 2.0 * k * k * k / 3.0);
      }

      // records for the boxes that have redundant points
      std::vector<BoxRec<T>> recs;
      std::vector<int> clsidx;
      int max_k = 0, max_r = 0, max_c = 0;
      for (int q = 0; q < nb; ++q) {
        const int B = boxes[q], bx = B % g, by = B / g;
        const int k = hk[q], n = cur.n[B], r = n - k;
        info.k[B] = k;
        if (r <= 0) continue;
        int c = k;
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (!dx && !dy) continue;
            const int x = bx + dx, y = by + dy;
            if (x < 0 || y < 0 || x >= g || y >= g) continue;
            c += cur.nact[y * g + x];
          }
        BoxRec<T> R{};
        R.box = B; R.k = k; R.r = r; R.c = c;
        R.Tm = static_cast<T*>(f->arena.get(sizeof(T) * (size_t)k * r));
        R.LU = static_cast<T*>(f->arena.get(sizeof(T) * (size_t)r * r));
        R.piv = static_cast<int*>(f->arena.get(sizeof(int) * r));
        R.LiP = static_cast<T*>(f->arena.get(sizeof(T) * (size_t)r * r));
        R.Ui = static_cast<T*>(f->arena.get(sizeof(T) * (size_t)r * r));
        R.Li = static_cast<T*>(f->arena.get(sizeof(T) * (size_t)r * r));
        R.E = static_cast<T*>(f->arena.get(sizeof(T) * (size_t)c * r));
        R.Ft = static_cast<T*>(f->arena.get(sizeof(T) * (size_t)c * r));
        R.idxR = static_cast<int*>(f->arena.get(sizeof(int) * r));
        R.idxC = static_cast<int*>(f->arena.get(sizeof(int) * c));
        R.cmap = static_cast<int*>(f->arena.get(sizeof(int) * c));
        if (!R.Tm || !R.LU || !R.piv || !R.LiP || !R.Ui || !R.Li || !R.E || !R.Ft || !R.idxR || !R.idxC ||
            !R.cmap) {
          rss_set_error("rss_factor: device arena allocation failed");
          return RSS_ENOMEM;
        }
        recs.push_back(R);
        clsidx.push_back(q);
        {
          const double cf = sizeof(T) == sizeof(double) ? 1.0 : 4.0;
          const double K = k, Rr = r, Cc = c;
          f->f_elim += cf * (4.0 * Cc * K * Rr + 4.0 * Rr * Rr * K + 2.0 * Rr * Rr * Rr / 3.0 + 2.0 * Cc * Rr * Rr);
          f->f_schur += cf * 2.0 * Cc * Cc * Rr;
        }
        max_k = std::max(max_k, k); max_r = std::max(max_r, r); max_c = std::max(max_c, c);
      }
      for (int q = 0; q < nb; ++q)
        if (cur.n[boxes[q]] - hk[q] > 0) cur.nact[boxes[q]] = hk[q];
      if (recs.empty()) continue;
      // a box may have c = 0 (rank 0 and no active neighbour: a far field that is
      // exactly zero); grids are sized for at least one row chunk, and the kernels
      // skip the chunks past each box's own c
      max_c = std::max(max_c, 1);
      const int nrec = (int)recs.size();
      // panel kernel shape: the widest panel (16 MA rows) whose shared memory
      // leaves room for two CTAs per SM; boxes beyond 200 KB take the row path
      int pan_ma = 1;
      size_t pan_max = 0;
      {
        int max_n = 0;
        for (const BoxRec<T>& R : recs) max_n = std::max(max_n, R.k + R.r);
        for (int ma : {4, 2, 1})
          if (panel_smem_bytes<T>(ma, max_n, max_r) <= 110 * 1024) { pan_ma = ma; break; }
        for (BoxRec<T>& R : recs) {
          const size_t pb = panel_smem_bytes<T>(pan_ma, R.k + R.r, R.r);
          R.panels = pb <= 200 * 1024 ? 1 : 0;
        }
      }
      // E = A_CB W_E and F^T = A_BC^T W_F on the tensor cores: real factors,
      // n <= 128 (the slices of a 64-row panel and of 32 columns of W fit in
      // shared memory)
      // (complex factors: any n_B, K taken in chunks by k_elim_ozc)
      int ozp_np = 0;
      const int ozp_nmax = sizeof(T) == sizeof(double) ? 128 : (1 << 30);
      // (real factors also keep the digit slices of the columns of W_E and W_F)
      auto wsl_bytes = [&](const BoxRec<T>& R) -> size_t {
        if (sizeof(T) != sizeof(double)) return 0;
        const size_t np = (R.k + R.r + 15) & ~15, rp = (R.r + 31) & ~31;
        return ((2 * rp * OZ_S * np * sizeof(uint16_t) + 255) & ~size_t(255)) + ((2 * rp * sizeof(int) + 255) & ~size_t(255));
      };
      if (prm->schur_path == 0 || prm->schur_path == 2) {
        size_t bytes = 0;
        for (const BoxRec<T>& R : recs)
          if (R.k + R.r <= ozp_nmax)
            bytes += 2 * (((size_t)(R.k + R.r) * R.r * sizeof(T) + 255) & ~size_t(255)) + wsl_bytes(R);
        if (bytes > 0) {
          if (!gb_w.ensure(bytes)) {
            rss_set_error("rss_factor: device workspace allocation failed");
            return RSS_ENOMEM;
          }
          char* p = static_cast<char*>(gb_w.p);
          for (BoxRec<T>& R : recs) {
            if (R.k + R.r > ozp_nmax) continue;
            const size_t b = ((size_t)(R.k + R.r) * R.r * sizeof(T) + 255) & ~size_t(255);
            R.We = reinterpret_cast<T*>(p);
            R.Wf = reinterpret_cast<T*>(p + b);
            p += 2 * b;
            if (sizeof(T) == sizeof(double)) {
              const size_t np = (R.k + R.r + 15) & ~15, rp = (R.r + 31) & ~31;
              const size_t bs = (2 * rp * OZ_S * np * sizeof(uint16_t) + 255) & ~size_t(255);
              R.Wsl = reinterpret_cast<uint16_t*>(p);
              R.Wexp = reinterpret_cast<int*>(p + bs);
              p += wsl_bytes(R);
            }
            R.ozp = 1;
            ozp_np = std::max(ozp_np, (R.k + R.r + 15) & ~15);
          }
          f->peak_transient = std::max(f->peak_transient, transient + bytes);
        }
      }
      for (const BoxRec<T>& R : recs)
        if (R.panels && !R.ozp) pan_max = std::max(pan_max, panel_smem_bytes<T>(pan_ma, R.k + R.r, R.r));
      // tensor-core Schur update for any r (K taken in chunks of 32)
      const bool oz = prm->schur_path == 0 || prm->schur_path == 2;
      const int ns = sizeof(T) == sizeof(double) ? OZ_S : 2 * OZ_S;   // slices per row
      int kp_max = 0;
      if (oz) {
        size_t bytes = 0;
        for (const BoxRec<T>& R : recs) {
          const int kp = (R.r + 15) & ~15;
          bytes += 2 * ((size_t)R.c * ns * kp * sizeof(uint16_t) + 256) + 2 * ((size_t)R.c * sizeof(int) + 256);
        }
        if (!gb_oz.ensure(bytes)) {
          rss_set_error("rss_factor: device workspace allocation failed");
          return RSS_ENOMEM;
        }
        char* p = static_cast<char*>(gb_oz.p);
        auto take = [&](size_t b) {
          char* q = p;
          p += (b + 255) & ~size_t(255);
          return q;
        };
        for (BoxRec<T>& R : recs) {
          R.kp = (R.r + 15) & ~15;
          kp_max = std::max(kp_max, R.kp);
          R.Esl = reinterpret_cast<uint16_t*>(take((size_t)R.c * ns * R.kp * sizeof(uint16_t)));
          R.Fsl = reinterpret_cast<uint16_t*>(take((size_t)R.c * ns * R.kp * sizeof(uint16_t)));
          R.Eexp = reinterpret_cast<int*>(take((size_t)R.c * sizeof(int)));
          R.Fexp = reinterpret_cast<int*>(take((size_t)R.c * sizeof(int)));
        }
        f->peak_transient = std::max(f->peak_transient, transient + bytes);
      }
      BoxRec<T>* d_recs = static_cast<BoxRec<T>*>(f->arena.get(sizeof(BoxRec<T>) * nrec));
      if (!d_recs) { rss_set_error("rss_factor: device arena allocation failed"); return RSS_ENOMEM; }
      RSS_CUDA(cudaMemcpyAsync(d_recs, recs.data(), sizeof(BoxRec<T>) * nrec, cudaMemcpyHostToDevice, st));
      RSS_CUDA(cudaMemcpyAsync(d_clsidx, clsidx.data(), sizeof(int) * nrec, cudaMemcpyHostToDevice, st));
      ElimArgs<T> ea;
      ea.L = cur.d;
      ea.recs = d_recs;
      ea.cls_idx = d_clsidx;
      ea.perm_in = d_perm;
      ea.T_ws = d_Tws;
      ea.err = d_err;
      ea.sym = (sizeof(T) == sizeof(double) && prm->kind == RSS_LAPLACE) ? 1 : 0;
      // shared memory of the per-box kernel: T and the LU of the largest box that fits
      const size_t ints = (2 * (size_t)max_r * sizeof(int) + 15) & ~size_t(15);
      const size_t want =
          sizeof(T) * ((size_t)max_r * max_r + std::max((size_t)max_k * max_r, (size_t)max_r * max_r)) + ints;
      const size_t ecap = std::min<size_t>(want, 200 * 1024);
      ea.smem_cap = (int)((ecap - ints) / sizeof(T));
      // the on-chip kernel when every box fits and takes E and F from the panel kernels
      size_t sm_lu = 0;
      bool lu_sm = true;
      for (const BoxRec<T>& R : recs) {
        sm_lu = std::max(sm_lu, elim_lu_sm_bytes<T>(R.k, R.r));
        lu_sm = lu_sm && (R.panels || R.ozp);
      }
      lu_sm = lu_sm && sm_lu <= 200 * 1024;
      evs.emplace_back(1, std::make_unique<Ev>());
      evs.back().second->start(st);
      if (lu_sm) {
        RSS_CUDA(cudaFuncSetAttribute(k_elim_lu_sm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_lu));
        k_elim_lu_sm<T><<<nrec, NT, sm_lu, st>>>(ea);
      } else {
        RSS_CUDA(cudaFuncSetAttribute(k_elim_lu<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ecap));
        k_elim_lu<T><<<nrec, NT, ecap, st>>>(ea);
      }
      RSS_LAUNCHED();
      if (pan_max > 0) {
        auto launch_panels = [&](auto kern, int rows) -> cudaError_t {
          cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pan_max);
          if (e != cudaSuccess) return e;
          kern<<<dim3((max_c + rows - 1) / rows, nrec), NT, pan_max, st>>>(ea);
          return cudaGetLastError();
        };
        RSS_CUDA(pan_ma == 4   ? launch_panels(k_elim_panels<T, 4>, 64)
                 : pan_ma == 2 ? launch_panels(k_elim_panels<T, 2>, 32)
                               : launch_panels(k_elim_panels<T, 1>, 16));
        RSS_LAUNCHED();
        f->launches += 1;
      }
      if constexpr (sizeof(T) == sizeof(double)) {
        if (ozp_np > 0) {
          k_w_split<<<nrec, NT, 0, st>>>(ea);
          RSS_LAUNCHED();
          const int smem = (64 + OZ_NCH) * (OZ_S * ozp_np + 8) * (int)sizeof(uint16_t);
          RSS_CUDA(cudaFuncSetAttribute(k_elim_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
          k_elim_oz<<<dim3((max_c + 63) / 64, nrec), NT, smem, st>>>(ea);
          RSS_LAUNCHED();
          f->launches += 2;
        }
      } else {
        if (ozp_np > 0) {
          const int smem = (ZCM + ZCN) * ZSA * (int)sizeof(uint16_t);
          RSS_CUDA(cudaFuncSetAttribute(k_elim_ozc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
          k_elim_ozc<<<dim3((max_c + ZCM - 1) / ZCM, nrec), NT, smem, st>>>(ea);
          RSS_LAUNCHED();
          f->launches += 1;
        }
      }
      evs.back().second->stop(st);
      const int ntile = (max_c + 63) / 64;
      evs.emplace_back(2, std::make_unique<Ev>());
      evs.back().second->start(st);
      if (oz) {
        if constexpr (sizeof(T) == sizeof(double)) {
          const int ntr_rows = (max_c + ST_M - 1) / ST_M;
          if (prm->schur_path == 0 && kp_max <= SRW_KP && (long long)nrec * ntr_rows >= 2 * 152) {
            // tcgen05, one CTA per 128-row block walking its column tiles (one CTA per SM)
            const int nchm = (kp_max + ST_KC - 1) / ST_KC;
            const int smem = std::max(nchm * ST_A + 2 * nchm * ST_B, 120 * 1024);
            RSS_CUDA(cudaFuncSetAttribute(k_schur_tc_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            k_schur_tc_rows<<<dim3(ntr_rows, nrec), SRW_NT, smem, st>>>(cur.d, d_recs, d_err, polls);
          } else if (prm->schur_path == 0 && kp_max <= 384) {   // tcgen05: FP32 group sums over the whole K
            const int smem = ST_A + ST_B;
            RSS_CUDA(cudaFuncSetAttribute(k_schur_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            const int ntr = (max_c + ST_M - 1) / ST_M, ntc = (max_c + ST_N - 1) / ST_N;
            k_schur_tc<<<dim3(ntr * ntc, nrec), ST_NT, smem, st>>>(cur.d, d_recs, d_err, polls);
          } else {
            const size_t smem = 2 * (size_t)SR_BUF * sizeof(uint16_t);
            RSS_CUDA(cudaFuncSetAttribute(k_schur_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            const int ntr = (max_c + SR_M - 1) / SR_M, ntc = (max_c + SR_N - 1) / SR_N;
            k_schur_oz<<<dim3(ntr * ntc, nrec), NT, smem, st>>>(cur.d, d_recs);
          }
        } else {
          if (prm->schur_path == 0 && kp_max <= 192) {   // tcgen05: Re/Im group sums exact for kp <= 192
            const int smem = SZ_A + 3 * SZ_B;
            RSS_CUDA(cudaFuncSetAttribute(k_schur_tc_c, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            const int ntr = (max_c + ST_M - 1) / ST_M, ntc = (max_c + ST_N - 1) / ST_N;
            k_schur_tc_c<<<dim3(ntr * ntc, nrec), ST_NT, smem, st>>>(cur.d, d_recs, d_err, polls);
          } else {
            const size_t smem = (64 + 32) * (size_t)SCSA * sizeof(uint16_t);
            RSS_CUDA(cudaFuncSetAttribute(k_schur_oz_c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            const int ntc = (max_c + 31) / 32;
            k_schur_oz_c<<<dim3(ntile * ntc, nrec), NT, smem, st>>>(cur.d, d_recs);
          }
        }
      } else {
        k_schur<T><<<dim3(ntile * ntile, nrec), NT, 0, st>>>(cur.d, d_recs);
      }
      RSS_LAUNCHED();
      evs.back().second->stop(st);
      for (BoxRec<T>& R : recs) R.Esl = R.Fsl = nullptr, R.Eexp = R.Fexp = nullptr;
      f->launches += 2;
      f->n_elim += 1;
      f->n_schur += 1;
      void* hcopy = std::malloc(sizeof(BoxRec<T>) * nrec);
      if (!hcopy) { rss_set_error("rss_factor: host allocation failed"); return RSS_ENOMEM; }
      std::memcpy(hcopy, recs.data(), sizeof(BoxRec<T>) * nrec);
      f->rec_host.push_back(hcopy);
      const int colour = (boxes[0] % g) % 3 + 3 * ((boxes[0] / g) % 3);
      f->batches.push_back(Batch{g, colour, nrec, d_recs, max_k, max_r, max_c});
    }
    RSS_CUDA(cudaStreamSynchronize(st));
    for (auto& pe : evs) {
      const double ms = pe.second->ms();
      (pe.first == 0 ? f->g_id : pe.first == 1 ? f->g_elim : f->g_schur) += ms;
      (pe.first == 0 ? info.g_id : pe.first == 1 ? info.g_elim : info.g_schur) += ms;
      (pe.first == 1 ? f->t_elim : pe.first == 2 ? f->t_schur : f->t_gen) += pe.first ? ms : 0.0;
    }
    int herr = 0;
    RSS_CUDA(cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr == RSS_ETIMEOUT) {
      rss_set_error("rss_factor: a tensor-core barrier wait of the Schur update ran out");
      return RSS_ETIMEOUT;
    }
    if (herr) { rss_set_error("rss_factor: zero pivot in the LU of a redundant block"); return RSS_ENUMERIC; }
    f->levels.push_back(info);

    // merge to the parent level
    Timer tm;
    const int gp = g / 2;
    HostLevel<T> par;
    par.n.assign(gp * gp, 0);
    int pmax = 1;
    for (int Pb = 0; Pb < gp * gp; ++Pb) {
      const int px = Pb % gp, py = Pb / gp;
      int s = 0;
      for (int q = 0; q < 4; ++q) s += cur.nact[(2 * py + q / 2) * g + 2 * px + q % 2];
      par.n[Pb] = s;
      pmax = std::max(pmax, s);
    }
    if (pmax > 65535) { rss_set_error("rss_factor: box too large after merging"); return RSS_EINVAL; }
    par.nact = par.n;
    {
      // when the parent's blocks do not fit beside the child's, keep only the
      // child's active entries (all the merge reads) and free the rest first
      size_t fr = 0, tot = 0;
      RSS_CUDA(cudaMemGetInfo(&fr, &tot));
      fr += pool_idle_bytes();
      const size_t pbytes = sizeof(T) * (size_t)gp * gp * 25 * (size_t)pmax * pmax;
      if (pbytes + (size_t(4) << 30) > fr) {
        int kmax = 1;
        for (int b = 0; b < nbox; ++b) kmax = std::max(kmax, cur.nact[b]);
        const size_t cbytes = sizeof(T) * (size_t)nbox * 25 * (size_t)kmax * kmax;
        T* cblk = nullptr;
        int *cpts = nullptr, *cact = nullptr;
        if (pool_malloc(reinterpret_cast<void**>(&cblk), cbytes, st) != cudaSuccess ||
            pool_malloc(reinterpret_cast<void**>(&cpts), sizeof(int) * (size_t)nbox * kmax, st) != cudaSuccess ||
            pool_malloc(reinterpret_cast<void**>(&cact), sizeof(int) * (size_t)nbox * kmax, st) != cudaSuccess) {
          pool_free(cblk, st); pool_free(cpts, st); pool_free(cact, st);
          rss_set_error("rss_factor: out of device memory for the compacted child blocks");
          return RSS_ENOMEM;
        }
        k_compact_blk<T><<<nbox * 25, NT, 0, st>>>(cur.d, cblk, cpts, kmax);
        RSS_LAUNCHED();
        k_iota_rows<<<1024, NT, 0, st>>>(cact, nbox, kmax);
        RSS_LAUNCHED();
        RSS_CUDA(cudaStreamSynchronize(st));
        f->launches += 2;
        pool_free(cur.d.blk, st);
        pool_free(cur.d.pts, st);
        pool_free(cur.d.act, st);
        transient -= sizeof(T) * (size_t)nbox * 25 * nn;
        transient += cbytes;
        cur.d.blk = cblk;
        cur.d.pts = cpts;
        cur.d.act = cact;
        cur.d.nmax = kmax;
      }
    }
    LevelGuard<T> par_guard{par, st};
    {
      rss_status s = alloc_level(par, gp, pmax, transient, st);
      if (s != RSS_OK) return s;
    }
    f->peak_transient = std::max(f->peak_transient, transient);
    Ev evm;
    evm.start(st);
    k_merge_pts<T><<<gp * gp, NT, 0, st>>>(cur.d, par.d);
    RSS_LAUNCHED();
    {
      const size_t msmem = (size_t)par.d.nmax * (2 * sizeof(int) + 2 * sizeof(int2));
      if (msmem > 48 * 1024)
        RSS_CUDA(cudaFuncSetAttribute(k_merge_blk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem));
      k_merge_blk<T><<<gp * gp * 25, NT, msmem, st>>>(cur.d, par.d, d_ixy, d_tab, f->kp, side);
    }
    RSS_LAUNCHED();
    evm.stop(st);
    RSS_CUDA(cudaStreamSynchronize(st));
    f->g_merge += evm.ms();
    f->launches += 2;
    transient -= sizeof(T) * (size_t)nbox * 25 * (size_t)cur.d.nmax * cur.d.nmax;
    free_level(cur, st);
    cur = par;
    par.d = LevelDev<T>{};   // owned by cur from here
    g = gp;
    f->t_merge += tm.ms();
  }

  // dense LU of everything still active (box grid side <= 2)
  Timer tt;
  {
    const int nbox = g * g;
    int offs[5] = {0, 0, 0, 0, 0};
    for (int b = 0; b < nbox; ++b) offs[b + 1] = offs[b] + cur.n[b];
    for (int b = nbox + 1; b < 5; ++b) offs[b] = offs[nbox];
    const int ntop = offs[nbox];
    f->ntop = ntop;
    f->d_top_lu = f->arena.get(sizeof(T) * (size_t)ntop * ntop);
    f->d_top_piv = static_cast<int*>(f->arena.get(sizeof(int) * ntop));
    f->d_top_idx = static_cast<int*>(f->arena.get(sizeof(int) * ntop));
    f->d_top_inv = f->arena.get(sizeof(T) * (size_t)ntop * ntop);
    if (!f->d_top_lu || !f->d_top_piv || !f->d_top_idx || !f->d_top_inv) {
      rss_set_error("rss_factor: device arena allocation failed");
      return RSS_ENOMEM;
    }
    Ev evt;
    evt.start(st);
    k_top_assemble<T><<<nbox * nbox, NT, 0, st>>>(cur.d, static_cast<T*>(f->d_top_lu), ntop, f->d_top_idx,
                                                  make_int4(offs[0], offs[1], offs[2], offs[3]), offs[4]);
    RSS_LAUNCHED();
    for (int jb = 0; jb < ntop; jb += LB) {
      T* A = static_cast<T*>(f->d_top_lu);
      k_lu_panel<T><<<1, 1024, 0, st>>>(A, ntop, jb, f->d_top_piv, d_err);
      RSS_LAUNCHED();
      const int others = ntop - std::min(LB, ntop - jb);
      if (others > 0) {
        k_lu_swap_trsm<T><<<cdiv(others, 128), 128, 0, st>>>(A, ntop, jb, f->d_top_piv);
        RSS_LAUNCHED();
      }
      const int m = ntop - std::min(ntop, jb + LB);
      if (m > 0) {
        const int nt = (m + 63) / 64;
        k_lu_update<T><<<nt * nt, NT, 0, st>>>(A, ntop, jb);
        RSS_LAUNCHED();
      }
      f->launches += 3;
    }
    if (ntop > 0) {
      rss_status si = top_inverse<T>(static_cast<const T*>(f->d_top_lu), f->d_top_piv, ntop,
                                     static_cast<T*>(f->d_top_inv), st);
      if (si != RSS_OK) return si;
      f->launches += 3;
    }
    evt.stop(st);
    span.stop(st);
    f->launches += 1;
    RSS_CUDA(cudaStreamSynchronize(st));
    f->g_top += evt.ms();
    f->g_span = span.ms();
    f->f_top += (sizeof(T) == sizeof(double) ? 1.0 : 4.0) * (2.0 / 3.0 + 2.0) * (double)ntop * ntop * ntop;
    free_level(cur, st);
    int herr = 0;
    RSS_CUDA(cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) { rss_set_error("rss_factor: zero pivot in the dense top LU"); return RSS_ENUMERIC; }
  }
  f->t_top += tt.ms();
  {
    const rss_status sb = build_sweep_classes<T>(f, st);
    if (sb != RSS_OK) return sb;
  }
  f->t_total = total.ms();
  return RSS_OK;
}

template rss_status factor_impl<double>(const rss_tree*, const rss_params*, cudaStream_t, rss_factorization*);
template rss_status factor_impl<zd>(const rss_tree*, const rss_params*, cudaStream_t, rss_factorization*);
