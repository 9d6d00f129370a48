// Complex digit-slice GEMM on the bf16 tensor cores (warp-level MMAs), shared by
// the complex elimination panels and the complex multi-RHS sweeps.
#pragma once
#include "common.cuh"

// C(i, q) = sum_l A(i, l) B(l, q) for complex A (M x K) and B (K x 32): every row
// of A and column of B is scaled by one power of two for its real and imaginary
// parts and cut into eight 7-bit digit slices each (slices 0-7 real, 8-15
// imaginary); Re = Ar Br - Ai Bi and Im = Ar Bi + Ai Br are summed exactly per
// K chunk of 32 (bf16 MMAs, FP32 accumulators, the sign of Ai flipped on the
// fragment bits), gathered in int64 and added over the chunks in FP64.  Rows in
// tiles of 64; every thread of the CTA calls it.
constexpr int ZCN = 32, ZCM = 64, ZCK = 32, ZSA = 16 * ZCK + 8;

template <typename AF, typename BF, typename OF>
__device__ void tc_gemm_c(int M, int K, AF aval, BF bval, OF cout, uint16_t* As, uint16_t* Bs, int* rexp, int* cexp) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, t4 = lane & 3;
  const int m0 = (warp >> 1) * 16, n0 = (warp & 1) * 16;
  const int a_row = lane & 15, a_k = (lane >> 4) * 8;
  const int b_row = ((lane >> 4) << 3) + (lane & 7), b_k = ((lane >> 3) & 1) * 8;
  for (int mt = 0; mt < M; mt += ZCM) {
    double accr[2][4], acci[2][4];
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) accr[ni][e] = acci[ni][e] = 0.0;
    for (int kc = 0; kc < K; kc += ZCK) {
      const int kl = min(ZCK, K - kc);
      __syncthreads();
      {   // rows of A: 64 rows x 4 lanes
        const int row = tid >> 2, gl = tid & 3, i = mt + row;
        const bool act = i < M;
        unsigned long long mk = 0;
        if (act)
          for (int l = gl; l < kl; l += 4) {
            const zd v = aval(i, kc + l);
            mk = max(mk, max(oz_abs_bits(v.x), oz_abs_bits(v.y)));
          }
        mk = max(mk, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mk, 1));
        mk = max(mk, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mk, 2));
        const int eb = oz_emax_b(mk);
        if (gl == 0) rexp[row] = eb - 1022;
        uint16_t* dst = As + row * ZSA;
        for (int l = 2 * gl; l < ZCK; l += 8) {
          const zd v0 = (act && l < kl) ? aval(i, kc + l) : zd{0.0, 0.0};
          const zd v1 = (act && l + 1 < kl) ? aval(i, kc + l + 1) : zd{0.0, 0.0};
          uint32_t dr[8], di[8];
          oz_digits2(oz_scaled_int(v0.x, eb), oz_scaled_int(v1.x, eb), dr);
          oz_digits2(oz_scaled_int(v0.y, eb), oz_scaled_int(v1.y, eb), di);
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            *reinterpret_cast<uint32_t*>(dst + p * ZCK + l) = dr[p];
            *reinterpret_cast<uint32_t*>(dst + (8 + p) * ZCK + l) = di[p];
          }
        }
      }
      {   // columns of B: 32 columns x 8 lanes
        const int col = tid >> 3, gl = tid & 7;
        unsigned long long mk = 0;
        for (int l = gl; l < kl; l += 8) {
          const zd b = bval(kc + l, col);
          mk = max(mk, max(oz_abs_bits(b.x), oz_abs_bits(b.y)));
        }
#pragma unroll
        for (int d = 1; d < 8; d <<= 1)
          mk = max(mk, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mk, d));
        const int eb = oz_emax_b(mk);
        if (gl == 0) cexp[col] = eb - 1022;
        uint16_t* dst = Bs + col * ZSA;
        for (int l = 2 * gl; l < ZCK; l += 16) {
          const zd v0 = l < kl ? bval(kc + l, col) : zd{0.0, 0.0};
          const zd v1 = l + 1 < kl ? bval(kc + l + 1, col) : zd{0.0, 0.0};
          uint32_t dr[8], di[8];
          oz_digits2(oz_scaled_int(v0.x, eb), oz_scaled_int(v1.x, eb), dr);
          oz_digits2(oz_scaled_int(v0.y, eb), oz_scaled_int(v1.y, eb), di);
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            *reinterpret_cast<uint32_t*>(dst + p * ZCK + l) = dr[p];
            *reinterpret_cast<uint32_t*>(dst + (8 + p) * ZCK + l) = di[p];
          }
        }
      }
      __syncthreads();
      long long Wr[2][4], Wi[2][4];
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int e = 0; e < 4; ++e) Wr[ni][e] = Wi[ni][e] = 0;
#pragma unroll 1
      for (int u = 0; u < 8; u += 2) {   // groups u, u + 1 together (|G| < 2^22)
        float cr0[2][4], ci0[2][4], cr1[2][4], ci1[2][4];
#pragma unroll
        for (int ni = 0; ni < 2; ++ni)
#pragma unroll
          for (int e = 0; e < 4; ++e) cr0[ni][e] = ci0[ni][e] = cr1[ni][e] = ci1[ni][e] = 0.f;
        for (int p = 0; p <= u + 1; ++p) {
          const uint16_t* Ar = As + p * ZCK + (m0 + a_row) * ZSA + a_k;
          const uint16_t* Ai = As + (8 + p) * ZCK + (m0 + a_row) * ZSA + a_k;
#pragma unroll
          for (int kk = 0; kk < ZCK; kk += 16) {
            uint32_t ar[4], ai[4], ain[4], br[4], bi[4];
            ldsm_x4(ar, Ar + kk);
            ldsm_x4(ai, Ai + kk);
#pragma unroll
            for (int i = 0; i < 4; ++i) ain[i] = ai[i] ^ 0x80008000u;
            ldsm_x4(br, Bs + (u + 1 - p) * ZCK + (n0 + b_row) * ZSA + b_k + kk);
            ldsm_x4(bi, Bs + (8 + u + 1 - p) * ZCK + (n0 + b_row) * ZSA + b_k + kk);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              mma_bf16(cr1[h], ar, br + 2 * h);
              mma_bf16(cr1[h], ain, bi + 2 * h);
              mma_bf16(ci1[h], ar, bi + 2 * h);
              mma_bf16(ci1[h], ai, br + 2 * h);
            }
            if (p <= u) {
              ldsm_x4(br, Bs + (u - p) * ZCK + (n0 + b_row) * ZSA + b_k + kk);
              ldsm_x4(bi, Bs + (8 + u - p) * ZCK + (n0 + b_row) * ZSA + b_k + kk);
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                mma_bf16(cr0[h], ar, br + 2 * h);
                mma_bf16(cr0[h], ain, bi + 2 * h);
                mma_bf16(ci0[h], ar, bi + 2 * h);
                mma_bf16(ci0[h], ai, br + 2 * h);
              }
            }
          }
        }
        const int sh = 32 - 7 * u;
#pragma unroll
        for (int ni = 0; ni < 2; ++ni)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const long long gr = (long long)(oz_fint(cr0[ni][e]) * 128 + oz_fint(cr1[ni][e]));
            const long long gi = (long long)(oz_fint(ci0[ni][e]) * 128 + oz_fint(ci1[ni][e]));
            Wr[ni][e] += sh >= 0 ? (gr << sh) : ((gr + (1LL << (-sh - 1))) >> (-sh));
            Wi[ni][e] += sh >= 0 ? (gi << sh) : ((gi + (1LL << (-sh - 1))) >> (-sh));
          }
      }
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int row = m0 + gq + (e >= 2 ? 8 : 0), col = n0 + ni * 8 + 2 * t4 + (e & 1);
          const int sx = rexp[row] + cexp[col] - 53;
          accr[ni][e] += oz_ldexp_int(Wr[ni][e], sx);
          acci[ni][e] += oz_ldexp_int(Wi[ni][e], sx);
        }
    }
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = m0 + gq + (e >= 2 ? 8 : 0), col = n0 + ni * 8 + 2 * t4 + (e & 1);
        if (mt + row < M) cout(mt + row, col, zd{accr[ni][e], acci[ni][e]});
      }
  }
  __syncthreads();
}
