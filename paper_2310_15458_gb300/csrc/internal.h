// Host-side objects behind the opaque rss_tree / rss_factor handles.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

constexpr int SWP_SPREAD_DEFAULT = 4;   // persistent sweeps: target work items per CTA and class

enum : uint32_t { RSS_TAG_TREE = 0x52545245u, RSS_TAG_FACTOR = 0x52464143u, RSS_TAG_SERVER = 0x52535256u };

// Quadtree over a uniform grid (Section 2.1).  Tree order: leaf boxes
// row-major over the leaf box grid, points row-major inside a leaf box.
struct rss_tree {
  uint32_t tag = RSS_TAG_TREE;
  int64_t n = 0;
  int side = 0;       // grid points per row
  int leaf = 0;       // points per leaf box
  int ls = 0;         // leaf box side in points
  int gL = 0;         // leaf box grid side
  Geo geo{};
  std::vector<int32_t> user_to_tree;  // tree index of each user point
  std::vector<int32_t> tree_to_user;
};

// One eliminated box (Eq. 8 / Eq. 9 record).  All pointers are device memory
// inside the factor's arena.  Matrices are column-major.
template <typename T> struct BoxRec {
  int box, k, r, c;
  T* Tm;        // k x r, ld k
  T* LU;        // r x r packed LU of X_RR, ld r
  int* piv;     // r getrf pivots (0-based)
  T* LiP;       // r x r, ld r: L_R^{-1} P_R (the solve applies it as one product)
  T* Ui;        // r x r, ld r: U_R^{-1}
  T* Li;        // r x r, ld r: L_R^{-1} (unit lower), factor time only
  int panels;   // 1: E and F^T are formed by the panel kernel
  T* E;         // c x r, ld c:  X_CR U_R^{-1}
  T* Ft;        // c x r, ld c:  (L_R^{-1} P_R X_RC)^T (plain transpose)
  int* idxR;    // r tree indices of R
  int* idxC;    // c tree indices of C = S then the neighbours' active points
  int* cmap;    // c entries (slot << 16 | position) used by the Schur update
  // factor-time only: E and F^T split into bf16 digit slices for the
  // tensor-core Schur update (null when the FP64 FMA kernel is used)
  uint16_t* Esl;  // c x (OZ_S * kp) bf16, row i at Esl + i * OZ_S * kp, slice p at + p * kp
  uint16_t* Fsl;
  int* Eexp;      // c row exponents
  int* Fexp;
  int kp;         // r rounded up to a multiple of 16
  // factor-time only, tensor-core panel path (ozp = 1): with the columns of B
  // in pivot order, E = A_CB W_E and F^T = A_BC^T W_F (n x r each, ld n), where
  // W_E = [-T U^{-1}; U^{-1}] and W_F = [-(L^{-1} P T^*)^T; (L^{-1} P)^T]
  T* We;
  T* Wf;
  // the columns of W_E then W_F (2 rp columns, rp = r rounded up to 32, the
  // padding columns zero), each cut into OZ_S bf16 digit slices of np = n
  // rounded up to 16 entries: column j at Wsl + j * OZ_S * np, slice p at
  // + p * np; Wexp[j] its power-of-two scale
  uint16_t* Wsl;
  int* Wexp;
  int ozp;
};


// Digit slices of the two large blocks of a real box record, for the
// tensor-core sweeps with many right-hand sides (built on first use): the rows
// of E (c rows, K = r) and the rows of F = (F^T)^T (r rows, K = c), each row cut
// into OZ_S bf16 digit slices under one power-of-two scale over its K entries.
struct SliceRec {
  uint16_t* Esl;   // c x OZ_S x kp: row i at Esl + i * OZ_S * kp, slice p at + p * kp
  int* Eexp;       // c row scales
  uint16_t* Fsl;   // r x OZ_S x cp
  int* Fexp;       // r row scales
  int kp, cp;      // r and c rounded up to 16 (zero padding)
};

struct Batch {
  int side;       // box grid side of the level
  int colour;
  int nrec;
  void* d_recs;   // BoxRec<T>[nrec] on the device
  int max_k, max_r, max_c;
};

struct LevelInfo {
  int side;
  std::vector<int32_t> n;   // points per box at level start
  std::vector<int32_t> k;   // skeleton rank per box
  double g_id = 0, g_elim = 0, g_schur = 0;   // device ms of the level's phases
};

// Stream-ordered device memory from the library's pool of the current device.
// Freed blocks stay reserved by the pool (release threshold: unlimited) until
// rss_trim_memory.  pool_malloc retries once after returning idle memory to the
// driver; it leaves *p null and the CUDA error state clear on failure.
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t st);
void pool_free(void* p, cudaStream_t st);   // stream-ordered; null is ignored
size_t pool_idle_bytes();                   // reserved by the pool but not in use

// Device memory arena: big chunks, bump allocation, freed together.  Chunks
// come from the pool in the order of stream `st` (the factor's stream).
struct Arena {
  std::vector<void*> chunks;
  char* cur = nullptr;
  size_t left = 0;
  size_t total = 0;
  size_t chunk_min = size_t(256) << 20;
  cudaStream_t st = nullptr;
  void* get(size_t bytes);   // nullptr on failure
  void release();            // waits for the device first
};

struct rss_factorization {
  uint32_t tag = RSS_TAG_FACTOR;
  bool is_complex = false;
  int64_t n = 0;
  int side = 0, leaf = 0, gL = 0;
  rss_params params{};
  KParams kp{};
  Geo geo{};
  int32_t* d_user_to_tree = nullptr;   // n
  int32_t* d_user_to_grid = nullptr;   // n: iy * side + ix of each user point (arena)
  double* d_w = nullptr;               // Lippmann-Schwinger weights per grid point (arena)
  void* mv = nullptr;                  // FFT matvec state (iterative.cu), built on first use
  std::vector<int32_t> tree_to_user;   // host copy, for inspection calls
  Arena arena;
  std::vector<Batch> batches;          // factor order
  void* d_swp = nullptr;               // the batches as the persistent sweeps read them (arena)
  int swp_spread = 0;                  // their schedule's knobs (0: the defaults; rss_tune_solve sets them):
  int swp_ctas = 0;                    // work items per CTA and class, CTAs per SM (0: as many as fit),
  int swp_launch = 0;                  // the launch form (0, 1: per-class kernels; 2: persistent;
                                       // 3: per-class, then persistent for the coarse tail),
  int swp_tail_boxes = 0;              // and the tail: the classes with fewer boxes than this
  std::vector<void*> rec_host;         // host copies of the BoxRec arrays (owned)
  std::vector<LevelInfo> levels;
  // top dense block
  int ntop = 0;
  void* d_top_lu = nullptr;            // ntop x ntop
  int* d_top_piv = nullptr;
  int* d_top_idx = nullptr;            // tree indices
  void* d_top_inv = nullptr;           // ntop x ntop: A_top^{-1}, applied by the solve
  // slices of E and F for the tensor-core sweeps (real factors), built by the
  // first solve that uses them: one pool block, one SliceRec array per batch
  std::mutex slice_mu;
  bool slices_ready = false;
  void* d_slice_mem = nullptr;
  size_t slice_bytes = 0;
  std::vector<SliceRec*> d_slices;
  // wall times (ms, host clock around each synchronised phase) for rss_info
  double t_gen = 0, t_id = 0, t_elim = 0, t_schur = 0, t_merge = 0, t_top = 0, t_total = 0;
  // device times (ms, CUDA events on the factor's stream), algorithmic real
  // flops (a complex multiply-add counts 8) and launch counts per phase
  double g_gen = 0, g_id = 0, g_elim = 0, g_schur = 0, g_merge = 0, g_top = 0;
  double g_span = 0;   // device time from the first kernel to the end of the top inverse
  double f_id = 0, f_elim = 0, f_schur = 0, f_top = 0;
  long long n_id = 0, n_elim = 0, n_schur = 0;
  long long launches = 0;
  size_t peak_transient = 0;
};

template <typename T> rss_status factor_impl(const rss_tree* tree, const rss_params* p,
                                             cudaStream_t st, rss_factorization* f);
template <typename T> rss_status solve_impl(const rss_factorization* f, T* b_dev, int64_t nrhs,
                                            int64_t ldb, cudaStream_t st);
template <typename T> rss_status top_inverse(const T* LU, const int* piv, int n, T* Ainv, cudaStream_t st);
// device bytes one solve of nrhs columns allocates (working copy plus sweep
// workspace), beside the caller's b
size_t solve_device_bytes(const rss_factorization* f, int64_t nrhs);
// the factor's colour classes as the persistent sweeps read them (arena, once)
template <typename T> rss_status build_sweep_classes(rss_factorization* f, cudaStream_t st);
// device bytes of the factor-owned caches that solves with up to max_nrhs
// columns build on first use (the digit slices of E and F of a real factor;
// 0 when none applies), and the call that builds them now, on st
size_t solve_cache_bytes(const rss_factorization* f, int64_t max_nrhs);
rss_status prepare_solve_caches(const rss_factorization* f, int64_t max_nrhs, cudaStream_t st);
void free_factor(rss_factorization* f);
void free_matvec(rss_factorization* f);
rss_status self_integral(int kind, double h, double kappa, double* re, double* im);
void free_server(rss_server* s);
