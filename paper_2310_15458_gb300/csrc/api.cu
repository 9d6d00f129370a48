// C ABI entry points: tree construction, dispatch on the scalar type,
// inspection, error reporting.  The numerical work lives in factor.cu and
// solve.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <sstream>

#include "internal.h"

static thread_local std::string g_last_error;

void rss_set_error(const std::string& msg) { g_last_error = msg; }

static rss_status fail(rss_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

// One pool per device, created on first use.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {};

static cudaError_t get_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}

cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = get_pool(&pool);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  if (bytes == 0) bytes = 256;
  e = cudaMallocFromPoolAsync(p, bytes, pool, st);
  if (e == cudaErrorMemoryAllocation) {
    // blocks freed on other streams may not be reusable yet: let them
    // complete, hand idle memory back to the driver, and try once more
    cudaGetLastError();
    cudaDeviceSynchronize();
    cudaMemPoolTrimTo(pool, 0);
    e = cudaMallocFromPoolAsync(p, bytes, pool, st);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
  }
  return e;
}

void pool_free(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

size_t pool_idle_bytes() {
  cudaMemPool_t pool = nullptr;
  if (get_pool(&pool) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  uint64_t reserved = 0, used = 0;
  cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
  cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
  return reserved > used ? (size_t)(reserved - used) : 0;
}

void* Arena::get(size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes == 0) bytes = 256;
  if (bytes > left) {
    size_t sz = std::max(bytes, chunk_min);
    void* p = nullptr;
    if (pool_malloc(&p, sz, st) != cudaSuccess) return nullptr;
    chunks.push_back(p);
    cur = static_cast<char*>(p);
    left = sz;
    total += sz;
  }
  void* out = cur;
  cur += bytes;
  left -= bytes;
  return out;
}

void Arena::release() {
  if (!chunks.empty()) cudaDeviceSynchronize();   // solves on any stream may still read the chunks
  for (void* p : chunks) pool_free(p, 0);
  chunks.clear();
  cur = nullptr;
  left = 0;
  total = 0;
}

extern "C" {

const char* rss_last_error(void) { return g_last_error.c_str(); }

rss_status rss_trim_memory(size_t keep_bytes) {
  cudaMemPool_t pool = nullptr;
  cudaError_t e = get_pool(&pool);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, keep_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(RSS_ECUDA, std::string("rss_trim_memory: ") + cudaGetErrorString(e));
  }
  return RSS_OK;
}

rss_status rss_build_tree(const double* pts, int64_t n, int leaf, rss_tree** out) {
  if (!out) return fail(RSS_EINVAL, "rss_build_tree: out is NULL");
  *out = nullptr;
  if (!pts || n <= 0) return fail(RSS_EINVAL, "rss_build_tree: no points");
  if (n > (int64_t(1) << 30)) return fail(RSS_EINVAL, "rss_build_tree: more than 2^30 points");
  int side = (int)std::llround(std::sqrt((double)n));
  if ((int64_t)side * side != n) return fail(RSS_EINVAL, "rss_build_tree: n is not a square");
  int ls = (int)std::llround(std::sqrt((double)leaf));
  if (leaf <= 0 || ls * ls != leaf || side % ls != 0)
    return fail(RSS_EINVAL, "rss_build_tree: leaf must be a square l*l with l dividing sqrt(n)");
  int gL = side / ls;
  if (gL & (gL - 1)) return fail(RSS_EINVAL, "rss_build_tree: sqrt(n)/sqrt(leaf) must be a power of two");
  if (leaf > 256) return fail(RSS_EINVAL, "rss_build_tree: leaf boxes hold at most 256 points");
  double xmin = pts[0], xmax = pts[0], ymin = pts[1], ymax = pts[1];
  for (int64_t i = 0; i < n; ++i) {
    double x = pts[2 * i], y = pts[2 * i + 1];
    if (!std::isfinite(x) || !std::isfinite(y)) return fail(RSS_EINVAL, "rss_build_tree: non-finite point");
    xmin = std::min(xmin, x); xmax = std::max(xmax, x);
    ymin = std::min(ymin, y); ymax = std::max(ymax, y);
  }
  double hg = side > 1 ? (xmax - xmin) / (side - 1) : 1.0;
  double hgy = side > 1 ? (ymax - ymin) / (side - 1) : 1.0;
  if (!(hg > 0) || std::fabs(hg - hgy) > 1e-9 * hg)
    return fail(RSS_EINVAL, "rss_build_tree: points do not span a square grid");
  rss_tree* t = new (std::nothrow) rss_tree();
  if (!t) return fail(RSS_ENOMEM, "rss_build_tree: host allocation failed");
  t->n = n; t->side = side; t->leaf = leaf; t->ls = ls; t->gL = gL;
  t->geo = Geo{xmin, ymin, hg, side};
  try {
    t->user_to_tree.assign(n, -1);
    t->tree_to_user.assign(n, -1);
  } catch (...) {
    delete t;
    return fail(RSS_ENOMEM, "rss_build_tree: host allocation failed");
  }
  for (int64_t i = 0; i < n; ++i) {
    double fx = (pts[2 * i] - xmin) / hg, fy = (pts[2 * i + 1] - ymin) / hg;
    long long ix = std::llround(fx), iy = std::llround(fy);
    if (ix < 0 || ix >= side || iy < 0 || iy >= side || std::fabs(fx - ix) > 1e-6 ||
        std::fabs(fy - iy) > 1e-6) {
      delete t;
      return fail(RSS_EINVAL, "rss_build_tree: a point is off the uniform grid");
    }
    int bx = (int)ix / ls, by = (int)iy / ls;
    int loc = (int)(iy % ls) * ls + (int)(ix % ls);
    int64_t ti = (int64_t)(by * gL + bx) * leaf + loc;
    if (t->tree_to_user[ti] != -1) {
      delete t;
      return fail(RSS_EINVAL, "rss_build_tree: two points share a grid node");
    }
    t->tree_to_user[ti] = (int32_t)i;
    t->user_to_tree[i] = (int32_t)ti;
  }
  *out = t;
  return RSS_OK;
}

rss_status rss_factor(const rss_tree* tree, const rss_params* p, void* stream, rss_factorization** out) {
  if (!out) return fail(RSS_EINVAL, "rss_factor: out is NULL");
  *out = nullptr;
  if (!tree || tree->tag != RSS_TAG_TREE) return fail(RSS_EINVAL, "rss_factor: not a tree handle");
  if (!p) return fail(RSS_EINVAL, "rss_factor: params is NULL");
  if (!(p->eps >= 0) || p->eps >= 1) return fail(RSS_EINVAL, "rss_factor: eps must be in [0, 1)");
  if (p->kind < RSS_LAPLACE || p->kind > RSS_HELMHOLTZ_LS) return fail(RSS_EINVAL, "rss_factor: unknown kernel kind");
  if (p->diag_rule != 0 && p->diag_rule != 1) return fail(RSS_EINVAL, "rss_factor: diag_rule must be 0 or 1");
  if (p->schur_path < 0 || p->schur_path > 2) return fail(RSS_EINVAL, "rss_factor: schur_path must be 0, 1 or 2");
  if ((p->kind == RSS_HELMHOLTZ || p->kind == RSS_HELMHOLTZ_LS) && !(p->kappa > 0))
    return fail(RSS_EINVAL, "rss_factor: the Helmholtz kernels need kappa > 0");
  if (p->diag_rule == 1 && (p->kind == RSS_TEST_POLY || p->kind == RSS_TEST_RPOLY))
    return fail(RSS_EINVAL, "rss_factor: diag_rule 1 needs a Laplace or Helmholtz kernel");
  if (p->proxy_n < 0 || p->proxy_n > 4096) return fail(RSS_EINVAL, "rss_factor: proxy_n out of range");
  if (p->ncoef < 0 || p->ncoef > RSS_MAX_COEF) return fail(RSS_EINVAL, "rss_factor: ncoef out of range");
  if (p->proxy_radius_over_side < 0) return fail(RSS_EINVAL, "rss_factor: negative proxy radius");
  if (p->wait_polls < -1) return fail(RSS_EINVAL, "rss_factor: wait_polls must be >= -1");
  int spread = 0, ctas = 0, launch = 0, tail = 0;
  if (p->tune_table) {   // the object rss_tune_solve writes: its last "launch", "spread", "ctas_per_sm"
    auto last = [&](const char* key) -> const char* {
      const char* hit = nullptr;
      for (const char* q = std::strstr(p->tune_table, key); q; q = std::strstr(q + 1, key)) hit = q;
      return hit ? std::strchr(hit, ':') : nullptr;
    };
    const char* l = last("\"launch\"");
    const char* v = l ? std::strchr(l, '"') : nullptr;
    launch = !v ? 2 : std::strncmp(v + 1, "per_class", 9) == 0 ? 1 : std::strncmp(v + 1, "hybrid", 6) == 0 ? 3 : 2;
    const char* q = last("\"spread\"");
    if (q) spread = std::atoi(q + 1);
    const char* tb = last("\"tail_boxes\"");
    tail = tb ? std::atoi(tb + 1) : 0;
    if (launch == 3 && tail < 1) return fail(RSS_EINVAL, "rss_factor: tune_table hybrid without tail_boxes >= 1");
    if (launch != 1 && (spread < 1 || spread > 1024))
      return fail(RSS_EINVAL, "rss_factor: tune_table has no \"spread\" between 1 and 1024");
    const char* c = last("\"ctas_per_sm\"");
    ctas = c ? std::atoi(c + 1) : 0;
    if (ctas < 0 || ctas > 64) return fail(RSS_EINVAL, "rss_factor: tune_table ctas_per_sm out of range");
  }
  rss_factorization* f = new (std::nothrow) rss_factorization();
  if (!f) return fail(RSS_ENOMEM, "rss_factor: host allocation failed");
  f->params = *p;
  f->params.tune_table = nullptr;   // read during this call only
  f->swp_spread = spread;
  f->swp_ctas = ctas;
  f->swp_launch = launch;
  f->swp_tail_boxes = tail;
  if (f->params.proxy_n == 0) f->params.proxy_n = 64;
  if (f->params.proxy_radius_over_side == 0) f->params.proxy_radius_over_side = 1.25;
  double h = p->h > 0 ? p->h : tree->geo.hg;
  f->kp.kind = p->kind;
  f->kp.h2 = h * h;
  f->kp.kappa = p->kappa;
  f->kp.diag_re = p->diag_re;
  f->kp.diag_im = p->diag_im;
  f->kp.ncoef = p->ncoef;
  for (int i = 0; i < RSS_MAX_COEF; ++i) {
    f->kp.cre[i] = p->coef_re[i];
    f->kp.cim[i] = p->coef_im[i];
  }
  f->kp.scale = p->scale;
  f->kp.phx = p->phase_x;
  f->kp.phy = p->phase_y;
  f->kp.w = nullptr;
  if (f->params.bump_a <= 0) {
    f->params.bump_cx = 0.5;
    f->params.bump_cy = 0.5;
    f->params.bump_a = 32.0;
  }
  if (p->diag_rule == 1) {   // the paper's self-cell quadrature (Eqs. 16, 20)
    double re = 0, im = 0;
    const rss_status si = self_integral(p->kind, h, p->kappa, &re, &im);
    if (si != RSS_OK) { delete f; return si; }
    f->kp.diag_re = re;
    f->kp.diag_im = im;
    f->params.diag_re = re;
    f->params.diag_im = im;
  }
  f->is_complex = (p->kind == RSS_HELMHOLTZ || p->kind == RSS_TEST_POLY || p->kind == RSS_HELMHOLTZ_LS);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rss_status s = f->is_complex ? factor_impl<zd>(tree, p, st, f) : factor_impl<double>(tree, p, st, f);
  if (s != RSS_OK) {
    std::string keep = g_last_error;
    cudaStreamSynchronize(st);
    cudaGetLastError();
    free_factor(f);
    g_last_error = keep;
    return s;
  }
  *out = f;
  return RSS_OK;
}

rss_status rss_solve(const rss_factorization* f, void* b, int64_t nrhs, int64_t ldb, void* stream) {
  if (!f || f->tag != RSS_TAG_FACTOR) return fail(RSS_EINVAL, "rss_solve: not a factor handle");
  if (!b) return fail(RSS_EINVAL, "rss_solve: b is NULL");
  if (nrhs <= 0) return fail(RSS_EINVAL, "rss_solve: nrhs must be positive");
  if (ldb < f->n) return fail(RSS_EINVAL, "rss_solve: ldb < n");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, b) != cudaSuccess) {
    cudaGetLastError();
    attr.type = cudaMemoryTypeUnregistered;
  }
  const size_t esz = f->is_complex ? 16 : 8;
  const bool on_device = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
  if (on_device) {
    return f->is_complex ? solve_impl<zd>(f, static_cast<zd*>(b), nrhs, ldb, st)
                         : solve_impl<double>(f, static_cast<double*>(b), nrhs, ldb, st);
  }
  // host buffer: stage through the device (copies inside this call)
  void* d = nullptr;
  size_t bytes = esz * (size_t)f->n * (size_t)nrhs;
  RSS_CUDA(pool_malloc(&d, bytes, st));
  rss_status s = RSS_OK;
  cudaError_t e = cudaMemcpy2DAsync(d, esz * f->n, b, esz * ldb, esz * f->n, nrhs,
                                    cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    s = f->is_complex ? solve_impl<zd>(f, static_cast<zd*>(d), nrhs, f->n, st)
                      : solve_impl<double>(f, static_cast<double*>(d), nrhs, f->n, st);
    if (s == RSS_OK)
      e = cudaMemcpy2DAsync(b, esz * ldb, d, esz * f->n, esz * f->n, nrhs, cudaMemcpyDeviceToHost, st);
  }
  pool_free(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(RSS_ECUDA, std::string("rss_solve: ") + cudaGetErrorString(e));
  return s;
}

void rss_free(void* h) {
  if (!h) return;
  uint32_t tag = *static_cast<uint32_t*>(h);
  if (tag == RSS_TAG_TREE) {
    rss_tree* t = static_cast<rss_tree*>(h);
    t->tag = 0;
    delete t;
  } else if (tag == RSS_TAG_FACTOR) {
    free_factor(static_cast<rss_factorization*>(h));
  } else if (tag == RSS_TAG_SERVER) {
    free_server(static_cast<rss_server*>(h));
  }
}

rss_status rss_info(const rss_factorization* f, char* buf, size_t len) {
  if (!f || f->tag != RSS_TAG_FACTOR || !buf || len == 0) return fail(RSS_EINVAL, "rss_info: bad arguments");
  std::ostringstream o;
  o << "{\"n\": " << f->n << ", \"complex\": " << (f->is_complex ? "true" : "false")
    << ", \"leaf\": " << f->leaf << ", \"ntop\": " << f->ntop
    << ", \"arena_bytes\": " << f->arena.total << ", \"peak_transient_bytes\": " << f->peak_transient
    << ", \"launches\": " << f->launches << ", \"batches\": " << f->batches.size()
    << ", \"solve_spread\": " << (f->swp_spread > 0 ? f->swp_spread : SWP_SPREAD_DEFAULT)
    << ", \"solve_ctas_per_sm\": " << f->swp_ctas
    << ", \"solve_launch\": \"" << (f->swp_launch == 2 ? "persistent" : f->swp_launch == 3 ? "hybrid" : "per_class")
    << "\", \"solve_tail_boxes\": " << f->swp_tail_boxes
    << ", \"ms\": {\"gen\": " << f->t_gen << ", \"id\": " << f->t_id << ", \"elim\": " << f->t_elim
    << ", \"schur\": " << f->t_schur << ", \"merge\": " << f->t_merge << ", \"top\": " << f->t_top
    << ", \"total\": " << f->t_total << "}, \"gpu_ms\": {\"gen\": " << f->g_gen << ", \"id\": " << f->g_id
    << ", \"elim\": " << f->g_elim << ", \"schur\": " << f->g_schur << ", \"merge\": " << f->g_merge
    << ", \"top\": " << f->g_top << ", \"span\": " << f->g_span << "}, \"flops\": {\"id\": " << f->f_id << ", \"elim\": " << f->f_elim
    << ", \"schur\": " << f->f_schur << ", \"top\": " << f->f_top << "}, \"phase_launches\": {\"id\": "
    << f->n_id << ", \"elim\": " << f->n_elim << ", \"schur\": " << f->n_schur << "}, \"levels\": [";
  for (size_t l = 0; l < f->levels.size(); ++l) {
    const LevelInfo& L = f->levels[l];
    long long sk = 0, sn = 0;
    int kmax = 0, kmin = 1 << 30, nmax = 0;
    for (size_t b = 0; b < L.k.size(); ++b) {
      sk += L.k[b]; sn += L.n[b];
      kmax = std::max(kmax, (int)L.k[b]); kmin = std::min(kmin, (int)L.k[b]);
      nmax = std::max(nmax, (int)L.n[b]);
    }
    o << (l ? ", " : "") << "{\"side\": " << L.side << ", \"k_mean\": " << (double)sk / L.k.size()
      << ", \"k_min\": " << kmin << ", \"k_max\": " << kmax << ", \"n_mean\": "
      << (double)sn / L.n.size() << ", \"n_max\": " << nmax << ", \"gpu_ms\": {\"id\": " << L.g_id
      << ", \"elim\": " << L.g_elim << ", \"schur\": " << L.g_schur << "}}";
  }
  o << "]}";
  std::string s = o.str();
  if (s.size() + 1 > len) return fail(RSS_EINVAL, "rss_info: buffer too small");
  std::memcpy(buf, s.c_str(), s.size() + 1);
  return RSS_OK;
}

rss_status rss_level_ranks(const rss_factorization* f, int side, int32_t* k_out) {
  if (!f || f->tag != RSS_TAG_FACTOR || !k_out) return fail(RSS_EINVAL, "rss_level_ranks: bad arguments");
  for (const LevelInfo& L : f->levels)
    if (L.side == side) {
      std::copy(L.k.begin(), L.k.end(), k_out);
      return RSS_OK;
    }
  return fail(RSS_EINVAL, "rss_level_ranks: no compressed level with that side");
}

}  // extern "C"

template <typename T>
static rss_status box_record_impl(const rss_factorization* f, int side, int box, int32_t* sizes, int64_t* S,
                                  int64_t* R, int64_t* C, void* Tm, void* LU, int32_t* piv, void* E,
                                  void* F) {
  for (size_t bi = 0; bi < f->batches.size(); ++bi) {
    const Batch& b = f->batches[bi];
    if (b.side != side) continue;
    const BoxRec<T>* recs = static_cast<const BoxRec<T>*>(f->rec_host[bi]);
    for (int i = 0; i < b.nrec; ++i) {
      const BoxRec<T>& r = recs[i];
      if (r.box != box) continue;
      int n = r.k + r.r;
      if (sizes) { sizes[0] = r.k; sizes[1] = r.r; sizes[2] = r.c; sizes[3] = n; }
      std::vector<int32_t> idx(std::max(r.c, r.r));
      auto to_user = [&](const int* d, int cnt, int64_t* dst) -> rss_status {
        if (!dst || cnt == 0) return RSS_OK;
        RSS_CUDA(cudaMemcpy(idx.data(), d, sizeof(int) * cnt, cudaMemcpyDeviceToHost));
        for (int q = 0; q < cnt; ++q) dst[q] = f->tree_to_user[idx[q]];
        return RSS_OK;
      };
      rss_status s;
      if ((s = to_user(r.idxC, r.k, S)) != RSS_OK) return s;
      if ((s = to_user(r.idxR, r.r, R)) != RSS_OK) return s;
      if ((s = to_user(r.idxC, r.c, C)) != RSS_OK) return s;
      if (Tm && r.k * r.r) RSS_CUDA(cudaMemcpy(Tm, r.Tm, sizeof(T) * r.k * r.r, cudaMemcpyDeviceToHost));
      if (LU) RSS_CUDA(cudaMemcpy(LU, r.LU, sizeof(T) * r.r * r.r, cudaMemcpyDeviceToHost));
      if (piv) RSS_CUDA(cudaMemcpy(piv, r.piv, sizeof(int) * r.r, cudaMemcpyDeviceToHost));
      if (E) RSS_CUDA(cudaMemcpy(E, r.E, sizeof(T) * r.c * r.r, cudaMemcpyDeviceToHost));
      if (F) {
        std::vector<T> ft((size_t)r.c * r.r);
        RSS_CUDA(cudaMemcpy(ft.data(), r.Ft, sizeof(T) * ft.size(), cudaMemcpyDeviceToHost));
        T* Fo = static_cast<T*>(F);   // r x c, ld r
        for (int i = 0; i < r.c; ++i)
          for (int j = 0; j < r.r; ++j) Fo[j + (size_t)i * r.r] = ft[i + (size_t)j * r.c];
      }
      return RSS_OK;
    }
  }
  return fail(RSS_EINVAL, "rss_box_record: box has no elimination record at that level");
}

extern "C" rss_status rss_box_record(const rss_factorization* f, int side, int box, int32_t* sizes, int64_t* S,
                                     int64_t* R, int64_t* C, void* Tm, void* LU, int32_t* piv,
                                     void* E, void* F) {
  if (!f || f->tag != RSS_TAG_FACTOR) return fail(RSS_EINVAL, "rss_box_record: not a factor handle");
  rss_status s = f->is_complex ? box_record_impl<zd>(f, side, box, sizes, S, R, C, Tm, LU, piv, E, F)
                               : box_record_impl<double>(f, side, box, sizes, S, R, C, Tm, LU, piv, E, F);
  return s;
}

void free_factor(rss_factorization* f) {
  if (!f) return;
  f->tag = 0;
  free_matvec(f);
  f->arena.release();   // waits for the device
  pool_free(f->d_slice_mem, 0);
  for (void* p : f->rec_host) std::free(p);
  delete f;
}
