// Block cyclic reduction factor and solve (see bcr.cuh for the algebra).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "bcr.cuh"
#include "tc_gemm.cuh"

namespace {

// ===================================================================== level 0
constexpr int TRI_WARPS = 2;

template <typename T>
__host__ __device__ size_t tri_smem_per_warp(int ny) {
  return ((size_t)6 * ny * sizeof(cplx<T>) + (size_t)ny + 15) & ~(size_t)15;
}

// Pivoted LU of the tridiagonal diagonal block T_r of an eliminated row r = 2k+1
// (Gaussian elimination with adjacent-row interchanges): multipliers dl, inverse
// pivots dinv, first and second superdiagonals du, du2 of U, and swap flags piv.
// One warp per row: the lanes stage the row's coefficients in shared memory, lane 0
// runs the sequential elimination there, and the lanes write the factors out.
template <typename T>
__global__ void __launch_bounds__(32 * TRI_WARPS)
tri_factor_kernel(const double2* __restrict__ dg, const double2* __restrict__ cy, int nx, int ny,
                  int m0, cplx<T>* __restrict__ tdl, cplx<T>* __restrict__ tdinv,
                  cplx<T>* __restrict__ tdu, cplx<T>* __restrict__ tdu2,
                  uint8_t* __restrict__ tpiv, int32_t* status) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * TRI_WARPS + w;
  if (k >= m0) return;  // whole warp
  cplx<T>* d = reinterpret_cast<cplx<T>*>(sm_raw + (size_t)w * tri_smem_per_warp<T>(ny));
  cplx<T>* o = d + ny;
  cplx<T>* dl = o + ny;
  cplx<T>* di = dl + ny;
  cplx<T>* du = di + ny;
  cplx<T>* du2 = du + ny;
  uint8_t* pv = reinterpret_cast<uint8_t*>(du2 + ny);
  const int64_t r = 2 * (int64_t)k + 1;
  for (int j = lane; j < ny; j += 32) {
    d[j] = ccast<T>(dg[r * ny + j]);
    o[j] = ccast<T>(cy[r * ny + j]);  // o[j] couples j and j+1
  }
  __syncwarp();
  if (lane == 0) {
    cplx<T> cur_d = d[0];
    cplx<T> cur_du = ny > 1 ? o[0] : czero<T>();
    bool sing = false;
    for (int j = 0; j < ny - 1; ++j) {
      const cplx<T> bs = o[j];
      const cplx<T> dnext = d[j + 1];
      const cplx<T> dunext = (j + 1 < ny - 1) ? o[j + 1] : czero<T>();
      if (cabs1(cur_d) >= cabs1(bs)) {
        if (cabs1(cur_d) == T(0)) sing = true;
        const cplx<T> inv = crecip(cur_d);
        const cplx<T> m = bs * inv;
        dl[j] = m;
        di[j] = inv;
        du[j] = cur_du;
        du2[j] = czero<T>();
        pv[j] = 0;
        cur_d = dnext - m * cur_du;
        cur_du = dunext;
      } else {
        const cplx<T> inv = crecip(bs);
        const cplx<T> m = cur_d * inv;
        dl[j] = m;
        di[j] = inv;
        du[j] = dnext;
        du2[j] = dunext;
        pv[j] = 1;
        cur_d = cur_du - m * dnext;
        cur_du = -(m * dunext);
      }
    }
    if (cabs1(cur_d) == T(0)) sing = true;
    di[ny - 1] = crecip(cur_d);
    dl[ny - 1] = czero<T>();
    du[ny - 1] = czero<T>();
    du2[ny - 1] = czero<T>();
    pv[ny - 1] = 0;
    if (sing) atomicCAS(status, DEV_OK, DEV_SINGULAR);
  }
  __syncwarp();
  const int64_t base = (int64_t)k * ny;
  for (int j = lane; j < ny; j += 32) {
    tdl[base + j] = dl[j];
    tdinv[base + j] = di[j];
    tdu[base + j] = du[j];
    tdu2[base + j] = du2[j];
    tpiv[base + j] = pv[j];
  }
}

template <typename T>
struct TriRow {
  const cplx<T>* dl;
  const cplx<T>* dinv;
  const cplx<T>* du;
  const cplx<T>* du2;
  const uint8_t* piv;
};

// Forward sweep (row interchanges and unit lower factor) for the right-hand side
// rhs(j), writing y_j through store(j, y).
template <typename T, typename Rhs, typename Store>
__device__ __forceinline__ void tri_forward(const TriRow<T>& f, int n, Rhs rhs, Store store) {
  cplx<T> cur = rhs(0);
  for (int j = 0; j < n - 1; ++j) {
    cplx<T> nb = rhs(j + 1);
    if (f.piv[j]) {
      store(j, nb);
      cur = cfms(f.dl[j], nb, cur);
    } else {
      store(j, cur);
      cur = cfms(f.dl[j], cur, nb);
    }
  }
  store(n - 1, cur);
}

// Backward substitution with U (diag, du, du2); load(j) returns y_j, emit(j, g_j).
template <typename T, typename Load, typename Emit>
__device__ __forceinline__ void tri_backward(const TriRow<T>& f, int n, Load load, Emit emit) {
  cplx<T> g1 = czero<T>(), g2 = czero<T>();  // g_{j+1}, g_{j+2}
#pragma unroll 4
  for (int j = n - 1; j >= 0; --j) {
    cplx<T> y = load(j);
    y = cfms(f.du[j], g1, y);
    y = cfms(f.du2[j], g2, y);
    cplx<T> g = y * f.dinv[j];
    emit(j, g);
    g2 = g1;
    g1 = g;
  }
}

// Forward sweep for the unit vector e_b into column ycol (stride ny).  Rows j < b - 1 of the
// sweep are exactly zero (the carried value stays zero until the unit entry is reached), so
// the sweep starts at row max(b - 1, 0) and writes only rows from there on; readers take the
// rows above as zero.
template <typename T>
__device__ __forceinline__ void tri_forward_unit(const TriRow<T>& f, int n, int b,
                                                 cplx<T>* ycol, int ny) {
  cplx<T> cur = b == 0 ? mkc(T(1), T(0)) : czero<T>();
  for (int j = b > 0 ? b - 1 : 0; j < n - 1; ++j) {
    const cplx<T> nb = (j + 1 == b) ? mkc(T(1), T(0)) : czero<T>();
    if (f.piv[j]) {
      ycol[(int64_t)j * ny] = nb;
      cur = cfms(f.dl[j], nb, cur);
    } else {
      ycol[(int64_t)j * ny] = cur;
      cur = cfms(f.dl[j], cur, nb);
    }
  }
  ycol[(int64_t)(n - 1) * ny] = cur;
}

// Dense Schur blocks of the first reduced system, one block per kept row e = 2k:
//   D'_k = T_e - diag(cx[e-1]) T_{e-1}^{-1} diag(cx[e-1]) - diag(cx[e]) T_{e+1}^{-1} diag(cx[e])
//   L'_k = -diag(cx[e-1]) T_{e-1}^{-1} diag(cx[e-2])
// Thread b forms column b of both inverses: the forward sweeps of the unit vector e_b go to
// two scratch columns (YR, YL: the next level's free working arrays; only the rows from
// b - 1 on, the others being zero), then one backward sweep runs both recurrences side by
// side, so that every entry of D'_k is formed in one step (no read-back of a partial D'),
// with the scratch loads issued a few rows ahead.
// MODE 1 forms instead the dense T_{2k+1}^{-1} of the eliminated rows k < m0 (the stored
// inverses of the solve with several right-hand sides), one block each, the forward sweep
// written in place into the output column: the backward sweep reads row a - PF before it
// writes row a, so every row is read before it is overwritten.
template <typename T, int MODE>
__global__ void level0_schur_kernel(const double2* __restrict__ dg, const double2* __restrict__ cx,
                                    const double2* __restrict__ cy, int nx, int ny,
                                    const cplx<T>* __restrict__ tdl, const cplx<T>* __restrict__ tdinv,
                                    const cplx<T>* __restrict__ tdu, const cplx<T>* __restrict__ tdu2,
                                    const uint8_t* __restrict__ tpiv, cplx<T>* __restrict__ Dn,
                                    cplx<T>* __restrict__ Ln, cplx<T>* scrR,
                                    cplx<T>* __restrict__ scrL, cplx<T>* G0) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(sm_raw);
  // [0,4ny): right factors, [4ny,8ny): left factors, then cxl2, cxl, cxr, dge, cye; piv bytes last
  cplx<T>* R = sm;
  cplx<T>* Lf = sm + 4 * ny;
  cplx<T>* cxl2 = sm + 8 * ny;
  cplx<T>* cxl = cxl2 + ny;
  cplx<T>* cxr = cxl + ny;
  cplx<T>* dge = cxr + ny;
  cplx<T>* cye = dge + ny;
  uint8_t* pivR = reinterpret_cast<uint8_t*>(cye + ny);
  uint8_t* pivL = pivR + ny;

  const int k = blockIdx.x;
  const int64_t e = 2 * (int64_t)k;
  const bool has_r = MODE == 1 || e + 1 < nx;   // eliminated row e+1 has index k
  const bool has_l = MODE == 0 && e >= 1;       // eliminated row e-1 has index k-1
  for (int j = threadIdx.x; j < ny; j += blockDim.x) {
    if (has_r) {
      int64_t b = (int64_t)k * ny + j;
      R[j] = tdl[b];
      R[ny + j] = tdinv[b];
      R[2 * ny + j] = tdu[b];
      R[3 * ny + j] = tdu2[b];
      pivR[j] = tpiv[b];
    }
    if (MODE == 1) continue;
    cxr[j] = has_r ? ccast<T>(cx[e * ny + j]) : czero<T>();
    if (has_l) {
      int64_t b = (int64_t)(k - 1) * ny + j;
      Lf[j] = tdl[b];
      Lf[ny + j] = tdinv[b];
      Lf[2 * ny + j] = tdu[b];
      Lf[3 * ny + j] = tdu2[b];
      pivL[j] = tpiv[b];
      cxl[j] = ccast<T>(cx[(e - 1) * ny + j]);
      cxl2[j] = ccast<T>(cx[(e - 2) * ny + j]);
    } else {
      cxl[j] = cxl2[j] = czero<T>();
    }
    dge[j] = ccast<T>(dg[e * ny + j]);
    cye[j] = ccast<T>(cy[e * ny + j]);
  }
  __syncthreads();
  const int b = threadIdx.x;
  if (b >= ny) return;
  const int64_t nn = (int64_t)ny * ny;
  cplx<T>* __restrict__ Dcol = Dn + (int64_t)k * nn + b;
  cplx<T>* __restrict__ Lcol = Ln + (int64_t)k * nn + b;
  cplx<T>* Gcol = G0 + (int64_t)k * nn + b;
  // MODE 1: the sweep in place in the output column
  cplx<T>* YR = MODE == 1 ? Gcol : scrR + (int64_t)k * nn + b;
  cplx<T>* __restrict__ YL = scrL + (int64_t)k * nn + b;
  const TriRow<T> fR{R, R + ny, R + 2 * ny, R + 3 * ny, pivR};
  const TriRow<T> fL{Lf, Lf + ny, Lf + 2 * ny, Lf + 3 * ny, pivL};
  if (has_r) tri_forward_unit<T>(fR, ny, b, YR, ny);
  if (has_l) tri_forward_unit<T>(fL, ny, b, YL, ny);
  const int a_lo = b > 0 ? b - 1 : 0;  // first row the sweeps wrote
  const cplx<T> sb = MODE == 0 ? cxr[b] : czero<T>();
  const cplx<T> sl = MODE == 0 ? cxl[b] : czero<T>();
  const cplx<T> sl2 = MODE == 0 ? cxl2[b] : czero<T>();
  cplx<T> r1 = czero<T>(), r2 = czero<T>(), l1 = czero<T>(), l2 = czero<T>();
  // scratch values of the next PF rows, loaded ahead of the recurrences
  constexpr int PF = 4;
  cplx<T> yr[PF], yl[PF];
#pragma unroll
  for (int q = 0; q < PF; ++q) {
    const int a = ny - 1 - q;
    yr[q] = (has_r && a >= a_lo) ? YR[(int64_t)a * ny] : czero<T>();
    yl[q] = (has_l && a >= a_lo) ? YL[(int64_t)a * ny] : czero<T>();
  }
  for (int a0 = ny - 1; a0 >= 0; a0 -= PF) {
#pragma unroll
    for (int q = 0; q < PF; ++q) {
      const int a = a0 - q;
      if (a < 0) break;
      const cplx<T> cr = yr[q], cl = yl[q];
      const int an = a - PF;  // the row PF steps ahead into the same ring slot
      yr[q] = (has_r && an >= a_lo) ? YR[(int64_t)an * ny] : czero<T>();
      yl[q] = (has_l && an >= a_lo) ? YL[(int64_t)an * ny] : czero<T>();
      // T_{e+1}^{-1} and T_{e-1}^{-1}, entry (a, b)
      cplx<T> gr = cfms(fR.du2[a], r2, cfms(fR.du[a], r1, cr)) * fR.dinv[a];
      if (!has_r) gr = czero<T>();
      r2 = r1;
      r1 = gr;
      if (MODE == 1) {
        Gcol[(int64_t)a * ny] = gr;
        continue;
      }
      cplx<T> gl = cfms(fL.du2[a], l2, cfms(fL.du[a], l1, cl)) * fL.dinv[a];
      if (!has_l) gl = czero<T>();
      l2 = l1;
      l1 = gl;
      const cplx<T> te = a == b ? dge[a] : (a == b - 1 ? cye[a] : (a == b + 1 ? cye[b] : czero<T>()));
      const cplx<T> cgl = cxl[a] * gl;
      Dcol[(int64_t)a * ny] = cfms(cgl, sl, cfms(cxr[a] * gr, sb, te));
      if (has_l) Lcol[(int64_t)a * ny] = -(cgl * sl2);
    }
  }
}

// shared memory of level0_schur_kernel: 13 ny complex values and 2 ny pivot flags
template <typename T>
inline size_t l0_smem(int ny) {
  return (size_t)13 * ny * sizeof(cplx<T>) + 2 * (size_t)ny;
}

// ===================================================================== Gauss-Jordan
// Blocked in-place inversion with partial pivoting (largest |re|+|im| in the column,
// ties to the lowest row).  For each panel of NB columns:
//   1. NB unblocked Gauss-Jordan steps restricted to the panel columns (row swaps of the
//      panel columns only, pivot rows scaled, other rows eliminated);
//   2. the panel's row swaps, in order, applied to every other column;
//   3. every other column updated at once by M, the product of the panel's elementary
//      Gauss-Jordan transforms: M differs from the identity only in the panel columns,
//      and the in-place algorithm leaves exactly M's columns there, so
//      A_rest <- M A_rest = A_rest + M[:, panel] A_rest[panel rows] off the panel rows and
//      M[panel, panel] A_rest[panel rows] on them (forming M - I there instead would cancel
//      catastrophically for diagonally dominant blocks, whose M_kk = 1/pivot).
// Row interchanges are undone as column interchanges on output.  One block of NT threads
// per matrix; the matrix lives in shared memory (SMEM) or in global memory (the source
// slot, which is destroyed); the panel rows of step 3 are staged in shared memory, and
// the column that feeds the next pivot search is kept contiguous (coln) so the search
// reads without bank conflicts.
constexpr size_t SMEM_LIMIT = 227 * 1024;

template <typename T>
struct GjSmem {
  // byte offsets of the shared-memory regions for an n x n matrix and panel width nb
  size_t coln, colk, rowk, tpanel, perm, idx, mat, total;
  __host__ __device__ GjSmem(int n, int nb, bool smem_matrix) {
    size_t e = sizeof(cplx<T>);
    coln = 0;
    colk = coln + (size_t)n * e;
    rowk = colk + (size_t)n * e;
    tpanel = rowk + (size_t)nb * e;
    perm = tpanel + (size_t)nb * n * e;
    idx = perm + (size_t)n * sizeof(int);
    mat = (idx + (size_t)n * sizeof(int) + 15) & ~(size_t)15;
    total = mat + (smem_matrix ? (size_t)n * n * e : 0);
  }
};

// NT threads = (NT/32) x 32; the update tiles are TR rows (stride NT/32) x TC columns
// (stride 32) per thread, so within a warp the panel-column reads broadcast and the
// staged-row reads are consecutive.
template <typename T, bool SMEM, int NB, int TR, int TC, int NT>
__global__ void __launch_bounds__(NT)
gj_inverse_kernel(cplx<T>* __restrict__ src, int64_t src_stride, cplx<T>* __restrict__ out,
                  int64_t out_stride, int n, int32_t* status) {
  static_assert((NB & (NB - 1)) == 0 && NB <= 32, "panel width: power of two <= 32");
  constexpr int TY = NT / 32;
  constexpr int LNB = NB == 32 ? 5 : NB == 16 ? 4 : NB == 8 ? 3 : NB == 4 ? 2 : NB == 2 ? 1 : 0;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const GjSmem<T> L(n, NB, SMEM);
  cplx<T>* coln = reinterpret_cast<cplx<T>*>(sm_raw + L.coln);    // column k before its swap
  cplx<T>* colk = reinterpret_cast<cplx<T>*>(sm_raw + L.colk);    // column k after the swap
  cplx<T>* rowk = reinterpret_cast<cplx<T>*>(sm_raw + L.rowk);    // scaled pivot row (panel)
  cplx<T>* tp = reinterpret_cast<cplx<T>*>(sm_raw + L.tpanel);    // panel rows, other columns
  int* perm = reinterpret_cast<int*>(sm_raw + L.perm);
  int* idx = reinterpret_cast<int*>(sm_raw + L.idx);
  __shared__ int s_p;
  __shared__ cplx<T> s_pinv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  cplx<T>* g = src + (int64_t)blockIdx.x * src_stride;
  cplx<T>* a = SMEM ? reinterpret_cast<cplx<T>*>(sm_raw + L.mat) : g;
  if (SMEM) {
    for (int e = tid; e < n * n; e += NT) a[e] = g[e];
  }
  bool sing = false;
  for (int c0 = 0; c0 < n; c0 += NB) {
    const int nb = n - c0 < NB ? n - c0 : NB;
    __syncthreads();
    for (int i = tid; i < n; i += NT) coln[i] = a[i * n + c0];
    __syncthreads();
    // ---------------- panel
    for (int k = c0; k < c0 + nb; ++k) {
      if (warp == 0) {
        T best = T(-1);
        int bi = k;
        for (int i = k + lane; i < n; i += 32) {
          T v = cabs1(coln[i]);
          if (v > best) {
            best = v;
            bi = i;
          }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          T ob = __shfl_down_sync(0xffffffffu, best, off);
          int oi = __shfl_down_sync(0xffffffffu, bi, off);
          if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
          }
        }
        if (lane == 0) {
          s_p = bi;
          if (!(best > T(0))) sing = true;
          s_pinv = crecip(coln[bi]);
          perm[k] = bi;
        }
      }
      __syncthreads();
      const int p = s_p;
      const cplx<T> pinv = s_pinv;
      for (int i = tid; i < n; i += NT) colk[i] = coln[i == k ? p : (i == p ? k : i)];
      if (tid < nb) {
        const int j = c0 + tid;
        cplx<T> rk = a[k * n + j];
        cplx<T> rp = a[p * n + j];
        cplx<T> v = (j == k ? mkc(T(1), T(0)) : rp) * pinv;
        if (p != k) a[p * n + j] = rk;
        a[k * n + j] = v;
        rowk[tid] = v;
      }
      __syncthreads();
      const int knext = k + 1 - c0;  // panel column whose new values feed the next pivot search
      const int kt = k - c0;
      for (int e = tid; e < (n << LNB); e += NT) {
        const int i = e >> LNB, t = e & (NB - 1);
        if (t >= nb) continue;
        const int j = c0 + t;
        if (i != k) {
          cplx<T> base = (t == kt) ? czero<T>() : a[i * n + j];
          cplx<T> v = cfms(colk[i], rowk[t], base);
          a[i * n + j] = v;
          if (t == knext) coln[i] = v;
        } else if (t == knext) {
          coln[i] = rowk[t];
        }
      }
      __syncthreads();
    }
    const int m = n - nb;
    if (m == 0) continue;
    // ---------------- panel row swaps on the other columns, in order; stage panel rows
    for (int jj = tid; jj < m; jj += NT) {
      const int j = jj < c0 ? jj : jj + nb;
      for (int t = 0; t < nb; ++t) {
        const int r = c0 + t, p = perm[r];
        if (p != r) {
          cplx<T> x = a[r * n + j];
          a[r * n + j] = a[p * n + j];
          a[p * n + j] = x;
        }
      }
    }
    __syncthreads();
    for (int t = 0; t < nb; ++t)
      for (int jj = tid; jj < m; jj += NT) {
        const int j = jj < c0 ? jj : jj + nb;
        tp[t * m + jj] = a[(c0 + t) * n + j];
      }
    __syncthreads();
    // ---------------- other columns (register tiles TR x TC)
    const int ty = warp, tx = lane;
    for (int r0 = 0; r0 < n; r0 += TY * TR) {
      for (int q0 = 0; q0 < m; q0 += 32 * TC) {
        cplx<T> acc[TR][TC];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
          for (int c = 0; c < TC; ++c) {
            const int i = r0 + ty + TY * r, jj = q0 + tx + 32 * c;
            const int j = jj < c0 ? jj : jj + nb;
            const bool panel_row = i >= c0 && i < c0 + nb;
            acc[r][c] = (i < n && jj < m && !panel_row) ? a[i * n + j] : czero<T>();
          }
        for (int t = 0; t < nb; ++t) {
          cplx<T> zv[TR], tv[TC];
#pragma unroll
          for (int r = 0; r < TR; ++r) {
            const int i = r0 + ty + TY * r;
            zv[r] = i < n ? a[i * n + c0 + t] : czero<T>();
          }
#pragma unroll
          for (int c = 0; c < TC; ++c) {
            const int jj = q0 + tx + 32 * c;
            tv[c] = jj < m ? tp[t * m + jj] : czero<T>();
          }
#pragma unroll
          for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) acc[r][c] = cfma(zv[r], tv[c], acc[r][c]);
        }
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
          for (int c = 0; c < TC; ++c) {
            const int i = r0 + ty + TY * r, jj = q0 + tx + 32 * c;
            const int j = jj < c0 ? jj : jj + nb;
            if (i < n && jj < m) a[i * n + j] = acc[r][c];
          }
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < n; ++j) idx[j] = j;
    for (int k = n - 1; k >= 0; --k) {
      int p = perm[k];
      int t = idx[k];
      idx[k] = idx[p];
      idx[p] = t;
    }
    if (sing) atomicCAS(status, DEV_OK, DEV_SINGULAR);
  }
  __syncthreads();
  cplx<T>* o = out + (int64_t)blockIdx.x * out_stride;
  for (int i = 0; i < n; ++i)
    for (int j = tid; j < n; j += NT) o[i * n + j] = a[i * n + idx[j]];
}

// Register-panel variant: the panel is NB = NT/32 columns wide and warp t holds panel
// column t in registers (lane L keeps rows L, L+32, ..., R slots).  A pivot step then
// costs one block barrier: after its own update, the warp that holds the next pivot
// column searches it (shuffles), publishes the swapped column, the pivot row index and
// 1/pivot to a double-buffered shared slot, and every warp updates its column from that
// slot and from shuffles of its own registers (rows k and p).  The update of the other
// columns after each panel is the one of gj_inverse_kernel.
template <typename T, int R>
__device__ __forceinline__ cplx<T> reg_select(const cplx<T> (&x)[R], int s) {
  cplx<T> v = x[0];
#pragma unroll
  for (int r = 1; r < R; ++r)
    if (s == r) v = x[r];
  return v;
}

template <typename T>
__device__ __forceinline__ cplx<T> shfl_c(cplx<T> v, int src) {
  return mkc(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// value held for row `row` by the warp (row = slot * 32 + lane)
template <typename T, int R>
__device__ __forceinline__ cplx<T> warp_row(const cplx<T> (&x)[R], int row) {
  return shfl_c<T>(reg_select<T, R>(x, row >> 5), row & 31);
}

// Pivot search on the warp's column (rows k..n-1), ties to the lowest row; publishes the
// column after the swap of rows k and p, p and 1/pivot.  Returns false if singular.
template <typename T, int R>
__device__ __forceinline__ bool gj_pivot(const cplx<T> (&x)[R], int k, int n, int lane,
                                         cplx<T>* colk, int* s_p, cplx<T>* s_pinv, int* perm) {
  T best = T(-1);
  int bi = k;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    if (i >= k && i < n) {
      T v = cabs1(x[r]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
  }
  if constexpr (sizeof(T) == 4) {
    // |re| + |im| >= 0, so its bit pattern orders like the value: the largest key over the
    // warp, then the lowest row holding it (a lane without rows has key 0 and row k, which
    // changes nothing: row k itself is a candidate whenever the maximum is 0)
    const uint32_t key = best >= T(0) ? __float_as_uint(best) : 0u;
    const uint32_t kmax = __reduce_max_sync(0xffffffffu, key);
    bi = (int)__reduce_min_sync(0xffffffffu, key == kmax ? (uint32_t)bi : 0xffffffffu);
    best = __uint_as_float(kmax);
  } else {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      T ob = __shfl_xor_sync(0xffffffffu, best, off);
      int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
  }
  const int p = bi;
  const cplx<T> vp = warp_row<T, R>(x, p), vk = warp_row<T, R>(x, k);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    if (i < n) colk[i] = i == k ? vp : (i == p ? vk : x[r]);
  }
  if (lane == 0) {
    *s_p = p;
    *s_pinv = crecip(vp);
    perm[k] = p;
  }
  return best > T(0);
}

template <typename T, bool SMEM, int R, int TR, int TC, int NT>
__global__ void __launch_bounds__(NT)
gj_regpanel_kernel(cplx<T>* __restrict__ src, int64_t src_stride, cplx<T>* __restrict__ out,
                   int64_t out_stride, int n, int32_t* status) {
  constexpr int NB = NT / 32;
  constexpr int TY = NT / 32;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const GjSmem<T> L(n, NB, SMEM);
  cplx<T>* const cbuf0 = reinterpret_cast<cplx<T>*>(sm_raw + L.coln);  // published pivot
  cplx<T>* const cbuf1 = reinterpret_cast<cplx<T>*>(sm_raw + L.colk);  // columns, alternating
  cplx<T>* tp = reinterpret_cast<cplx<T>*>(sm_raw + L.tpanel);
  int* perm = reinterpret_cast<int*>(sm_raw + L.perm);
  int* idx = reinterpret_cast<int*>(sm_raw + L.idx);
  __shared__ int s_p[2];
  __shared__ cplx<T> s_pinv[2];
  __shared__ int s_sing;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  cplx<T>* g = src + (int64_t)blockIdx.x * src_stride;
  cplx<T>* a = SMEM ? reinterpret_cast<cplx<T>*>(sm_raw + L.mat) : g;
  if (tid == 0) s_sing = 0;
  if (SMEM) {
    for (int e = tid; e < n * n; e += NT) a[e] = g[e];
  }
  for (int c0 = 0; c0 < n; c0 += NB) {
    const int nb = n - c0 < NB ? n - c0 : NB;
    const int t = warp, j = c0 + t;
    __syncthreads();
    cplx<T> x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = lane + 32 * r;
      x[r] = (t < nb && i < n) ? a[i * n + j] : czero<T>();
    }
    if (warp == 0 && !gj_pivot<T, R>(x, c0, n, lane, cbuf0, &s_p[0], &s_pinv[0], perm))
      s_sing = 1;
    __syncthreads();
    // ---------------- panel: one barrier per pivot
    for (int kt = 0; kt < nb; ++kt) {
      const int k = c0 + kt, b = kt & 1;
      if (t < nb) {
        const int p = s_p[b];
        const cplx<T> pinv = s_pinv[b];
        const cplx<T>* colk = b ? cbuf1 : cbuf0;
        const cplx<T> vp = warp_row<T, R>(x, p), vk = warp_row<T, R>(x, k);
        const cplx<T> rk = (t == kt ? mkc(T(1), T(0)) : vp) * pinv;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int i = lane + 32 * r;
          if (i < n) {
            const cplx<T> old = i == k ? vp : (i == p ? vk : x[r]);
            const cplx<T> base = t == kt ? czero<T>() : old;
            x[r] = i == k ? rk : cfms(colk[i], rk, base);
          }
        }
        if (t == kt + 1 &&
            !gj_pivot<T, R>(x, k + 1, n, lane, b ? cbuf0 : cbuf1, &s_p[b ^ 1], &s_pinv[b ^ 1],
                            perm))
          s_sing = 1;
      }
      __syncthreads();
    }
    if (t < nb) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
        if (i < n) a[i * n + j] = x[r];
      }
    }
    const int m = n - nb;
    if (m == 0) continue;
    // ---------------- panel row swaps on the other columns, in order; stage panel rows
    for (int jj = tid; jj < m; jj += NT) {
      const int jc = jj < c0 ? jj : jj + nb;
      for (int u = 0; u < nb; ++u) {
        const int rr = c0 + u, p = perm[rr];
        if (p != rr) {
          cplx<T> y = a[rr * n + jc];
          a[rr * n + jc] = a[p * n + jc];
          a[p * n + jc] = y;
        }
      }
    }
    __syncthreads();
    for (int u = 0; u < nb; ++u)
      for (int jj = tid; jj < m; jj += NT) {
        const int jc = jj < c0 ? jj : jj + nb;
        tp[u * m + jj] = a[(c0 + u) * n + jc];
      }
    __syncthreads();
    // ---------------- other columns (register tiles TR x TC)
    const int ty = warp, tx = lane;
    for (int r0 = 0; r0 < n; r0 += TY * TR) {
      for (int q0 = 0; q0 < m; q0 += 32 * TC) {
        cplx<T> acc[TR][TC];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
          for (int c = 0; c < TC; ++c) {
            const int i = r0 + ty + TY * r, jj = q0 + tx + 32 * c;
            const int jc = jj < c0 ? jj : jj + nb;
            const bool panel_row = i >= c0 && i < c0 + nb;
            acc[r][c] = (i < n && jj < m && !panel_row) ? a[i * n + jc] : czero<T>();
          }
        for (int u = 0; u < nb; ++u) {
          cplx<T> zv[TR], tv[TC];
#pragma unroll
          for (int r = 0; r < TR; ++r) {
            const int i = r0 + ty + TY * r;
            zv[r] = i < n ? a[i * n + c0 + u] : czero<T>();
          }
#pragma unroll
          for (int c = 0; c < TC; ++c) {
            const int jj = q0 + tx + 32 * c;
            tv[c] = jj < m ? tp[u * m + jj] : czero<T>();
          }
#pragma unroll
          for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) acc[r][c] = cfma(zv[r], tv[c], acc[r][c]);
        }
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
          for (int c = 0; c < TC; ++c) {
            const int i = r0 + ty + TY * r, jj = q0 + tx + 32 * c;
            const int jc = jj < c0 ? jj : jj + nb;
            if (i < n && jj < m) a[i * n + jc] = acc[r][c];
          }
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    for (int jx = 0; jx < n; ++jx) idx[jx] = jx;
    for (int k = n - 1; k >= 0; --k) {
      int p = perm[k];
      int y = idx[k];
      idx[k] = idx[p];
      idx[p] = y;
    }
    if (s_sing) atomicCAS(status, DEV_OK, DEV_SINGULAR);
  }
  __syncthreads();
  cplx<T>* o = out + (int64_t)blockIdx.x * out_stride;
  for (int i = 0; i < n; ++i)
    for (int jx = tid; jx < n; jx += NT) o[i * n + jx] = a[i * n + idx[jx]];
}

// Look-ahead variant for FP32 blocks held in shared memory (n <= 160), 1024 threads in
// two groups of 16 warps.  While the panel group factors panel P+1 (one named barrier per
// pivot), the trailing group applies the rank-nb update of panel P to every column outside
// panels P and P+1; the panel group has applied that update to its own columns first.
// Rows are never swapped: the pivot of column k is physical row piv[k], chosen among the
// rows not yet used as pivots, and the permutations are applied when the inverse is
// written out (inverse[i][j] = M[piv[i]][pinv[j]] for the in-place result M).  Every entry
// is formed by the same operations as with explicit swaps, so the result equals that of
// gj_regpanel_kernel whenever no two pivot candidates tie.  The matrix row stride is odd
// (n | 1 entries), so that a warp reading one column (rows lane, lane + 32, ...) meets no
// bank conflict.
constexpr int GJLA_THREADS = 1024, GJLA_NB = 16, GJLA_R = 5, GJLA_TR = 5, GJLA_TC = 2;

struct GjLaSmem {
  // byte offsets for an n x n complex-FP32 matrix (odd row stride n | 1)
  size_t cb0, cb1, tpanel, piv, rowpanel, pinv, mat, total;
  __host__ __device__ GjLaSmem(int n) {
    const size_t e = sizeof(float2);
    const size_t tmax = (size_t)GJLA_NB * (n > GJLA_NB ? n - GJLA_NB : 1);
    cb0 = 0;
    cb1 = cb0 + (size_t)n * e;
    tpanel = cb1 + (size_t)n * e;
    piv = tpanel + tmax * e;
    rowpanel = piv + (size_t)n * sizeof(int);
    pinv = rowpanel + (size_t)n * sizeof(int);
    mat = (pinv + (size_t)n * sizeof(int) + 15) & ~(size_t)15;
    total = mat + (size_t)n * (n | 1) * e;
  }
};

__device__ __forceinline__ void group_bar(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(GJLA_THREADS / 2) : "memory");
}

// Pivot of column k held by this warp (rows lane + 32 r, `used` marks rows already taken):
// the largest |re| + |im| among unused rows, ties to the lowest row; publishes the column,
// the row, 1/pivot, piv[k] and rowpanel[row] = c0.  Returns false if the column is zero
// on every unused row (or holds no number there).
__device__ __forceinline__ bool gjla_pivot(const float2 (&x)[GJLA_R], unsigned used, int k,
                                           int c0, int n, int lane, float2* colk, int* s_p,
                                           float2* s_pinv, int* piv, volatile int* rowpanel) {
  constexpr int R = GJLA_R;
  float best = -1.f;
  int bi = 0x7fffffff, first = 0x7fffffff;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    if (i < n) {
      colk[i] = x[r];
      if (!((used >> r) & 1u)) {
        const float v = cabs1(x[r]);
        if (first == 0x7fffffff) first = i;
        if (v > best) {
          best = v;
          bi = i;
        }
      }
    }
  }
  // |re| + |im| >= 0 orders like its bit pattern: the largest key over the warp, then the
  // lowest row holding it; a lane without a candidate offers key 0 and its first unused row
  if (best < 0.f) bi = first;
  const uint32_t key = best >= 0.f ? __float_as_uint(best) : 0u;
  const uint32_t kmax = __reduce_max_sync(0xffffffffu, key);
  const int p = (int)__reduce_min_sync(0xffffffffu, key == kmax ? (uint32_t)bi : 0xffffffffu);
  const float2 vp = warp_row<float, R>(x, p);
  if (lane == 0) {
    *s_p = p;
    *s_pinv = crecip(vp);
    piv[k] = p;
    rowpanel[p] = c0;
  }
  return __uint_as_float(kmax) > 0.f;
}

// Panel group: Gauss-Jordan steps on columns c0 .. c0+nb-1, warp t holding column c0 + t
// in x (rows lane + 32 r); the columns are written back to the matrix at the end.
__device__ __forceinline__ void gjla_panel(float2 (&x)[GJLA_R], int c0, int nb, int n, int ld,
                                           float2* a, float2* cbuf0, float2* cbuf1, int* s_p,
                                           float2* s_pinv, int* piv, volatile int* rowpanel,
                                           int* s_sing) {
  constexpr int R = GJLA_R;
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
  unsigned used = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    if (i >= n || rowpanel[i] >= 0) used |= 1u << r;
  }
  if (t == 0 && !gjla_pivot(x, used, c0, c0, n, lane, cbuf0, &s_p[0], &s_pinv[0], piv, rowpanel))
    *s_sing = 1;
  group_bar(1);
  for (int kt = 0; kt < nb; ++kt) {
    const int b = kt & 1;
    if (t < nb) {
      const int p = s_p[b];
      const float2 pinv = s_pinv[b];
      const float2* colk = b ? cbuf1 : cbuf0;
      if (lane == (p & 31)) used |= 1u << (p >> 5);
      if (t == kt) {
        // the pivot column becomes -column / pivot, and 1 / pivot on the pivot row
        const float2 rk = mkc(1.f, 0.f) * pinv;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int i = lane + 32 * r;
          if (i < n) x[r] = i == p ? rk : cfms(colk[i], rk, czero<float>());
        }
      } else {
        const float2 rk = warp_row<float, R>(x, p) * pinv;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int i = lane + 32 * r;
          if (i < n) x[r] = i == p ? rk : cfms(colk[i], rk, x[r]);
        }
      }
      if (t == kt + 1 && !gjla_pivot(x, used, c0 + kt + 1, c0, n, lane, b ? cbuf0 : cbuf1,
                                     &s_p[b ^ 1], &s_pinv[b ^ 1], piv, rowpanel))
        *s_sing = 1;
    }
    group_bar(1);
  }
  if (t < nb) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = lane + 32 * r;
      if (i < n) a[i * ld + c0 + t] = x[r];
    }
  }
}

__global__ void __launch_bounds__(GJLA_THREADS)
gj_lookahead_kernel(const float2* __restrict__ src, int64_t src_stride, float2* __restrict__ out,
                    int64_t out_stride, int n, int32_t* status) {
  constexpr int R = GJLA_R, NB = GJLA_NB, TR = GJLA_TR, TC = GJLA_TC, TY = 16;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const GjLaSmem L(n);
  float2* const cbuf0 = reinterpret_cast<float2*>(sm_raw + L.cb0);
  float2* const cbuf1 = reinterpret_cast<float2*>(sm_raw + L.cb1);
  float2* const tp = reinterpret_cast<float2*>(sm_raw + L.tpanel);
  int* const piv = reinterpret_cast<int*>(sm_raw + L.piv);
  // panel start at which the row became a pivot, -1 before: the trailing group reads it for
  // the rows of panel P while the panel group sets it for rows of panel P+1 (from -1 to
  // c0 + nb); either value differs from c0 of panel P, so the reading does not depend on
  // the order.  All accesses are volatile (relaxed), which makes the overlap well defined.
  volatile int* const rowpanel = reinterpret_cast<volatile int*>(sm_raw + L.rowpanel);
  int* const pinv = reinterpret_cast<int*>(sm_raw + L.pinv);
  float2* const a = reinterpret_cast<float2*>(sm_raw + L.mat);
  __shared__ int s_p[2];
  __shared__ float2 s_pinv[2];
  __shared__ int s_sing;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ld = n | 1;
  const bool panel_group = warp < 16;
  const float2* g = src + (int64_t)blockIdx.x * src_stride;
  if (tid == 0) s_sing = 0;
  for (int i = tid; i < n; i += GJLA_THREADS) rowpanel[i] = -1;
  for (int e = tid; e < n * n; e += GJLA_THREADS) {
    const int i = e / n, j = e - i * n;
    a[i * ld + j] = g[e];
  }
  __syncthreads();
  float2 x[R];
  if (panel_group) {
    const int nb0 = n < NB ? n : NB;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = lane + 32 * r;
      x[r] = (warp < nb0 && i < n) ? a[i * ld + warp] : czero<float>();
    }
    gjla_panel(x, 0, nb0, n, ld, a, cbuf0, cbuf1, s_p, s_pinv, piv, rowpanel, &s_sing);
  }
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += NB) {
    const int nb = n - c0 < NB ? n - c0 : NB;
    const int c1 = c0 + nb;                                 // next panel
    const int nb1 = n - c1 < NB ? n - c1 : NB;              // its width (0: none)
    if (n - nb == 0) break;
    if (panel_group) {
      if (nb1 > 0) {
        const int j = c1 + warp;
        if (warp < nb1) {
          // this column: the rank-nb update of panel P (its pivot rows start from zero)
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int i = lane + 32 * r;
            x[r] = (i < n && rowpanel[i] != c0) ? a[i * ld + j] : czero<float>();
          }
          for (int u = 0; u < nb; ++u) {
            const float2 tv = a[piv[c0 + u] * ld + j];
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const int i = lane + 32 * r;
              if (i < n) x[r] = cfma(a[i * ld + c0 + u], tv, x[r]);
            }
          }
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) x[r] = czero<float>();
        }
        gjla_panel(x, c1, nb1, n, ld, a, cbuf0, cbuf1, s_p, s_pinv, piv, rowpanel, &s_sing);
      }
    } else {
      // trailing group: columns q = 0 .. mt-1, matrix column jc(q), outside panels P, P+1
      const int tt = tid - GJLA_THREADS / 2, ty = warp - 16, tx = lane;
      const int mt = n - nb - nb1;
      for (int u = 0; u < nb; ++u) {
        const int pr = piv[c0 + u];
        for (int q = tt; q < mt; q += GJLA_THREADS / 2) {
          const int jc = q < c0 ? q : q + nb + nb1;
          tp[u * mt + q] = a[pr * ld + jc];
        }
      }
      group_bar(2);
      for (int r0 = 0; r0 < n; r0 += TY * TR) {
        bool prow[TR];
#pragma unroll
        for (int r = 0; r < TR; ++r) {
          const int i = r0 + ty + TY * r;
          prow[r] = i < n && rowpanel[i] == c0;
        }
        for (int q0 = 0; q0 < mt; q0 += 32 * TC) {
          float2 acc[TR][TC];
#pragma unroll
          for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) {
              const int i = r0 + ty + TY * r, q = q0 + tx + 32 * c;
              const int jc = q < c0 ? q : q + nb + nb1;
              acc[r][c] = (i < n && q < mt && !prow[r]) ? a[i * ld + jc] : czero<float>();
            }
          for (int u = 0; u < nb; ++u) {
            float2 zv[TR], tv[TC];
#pragma unroll
            for (int r = 0; r < TR; ++r) {
              const int i = r0 + ty + TY * r;
              zv[r] = i < n ? a[i * ld + c0 + u] : czero<float>();
            }
#pragma unroll
            for (int c = 0; c < TC; ++c) {
              const int q = q0 + tx + 32 * c;
              tv[c] = q < mt ? tp[u * mt + q] : czero<float>();
            }
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
              for (int c = 0; c < TC; ++c) acc[r][c] = cfma(zv[r], tv[c], acc[r][c]);
          }
#pragma unroll
          for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) {
              const int i = r0 + ty + TY * r, q = q0 + tx + 32 * c;
              const int jc = q < c0 ? q : q + nb + nb1;
              if (i < n && q < mt) a[i * ld + jc] = acc[r][c];
            }
        }
      }
    }
    __syncthreads();
  }
  for (int l = tid; l < n; l += GJLA_THREADS) pinv[piv[l]] = l;
  if (tid == 0 && s_sing) atomicCAS(status, DEV_OK, DEV_SINGULAR);
  __syncthreads();
  float2* o = out + (int64_t)blockIdx.x * out_stride;
  for (int e = tid; e < n * n; e += GJLA_THREADS) {
    const int i = e / n, jx = e - i * n;
    o[e] = a[piv[i] * ld + pinv[jx]];
  }
}

cudaError_t launch_gj_lookahead(const float2* src, int64_t src_stride, float2* out,
                                int64_t out_stride, int n, int batch, int32_t* status,
                                cudaStream_t s) {
  const GjLaSmem L(n);
  if (L.total > SMEM_LIMIT || n > 32 * GJLA_R) return cudaErrorInvalidValue;
  if (L.total > 48 * 1024)
    RCI_CUDA_TRY(cudaFuncSetAttribute(gj_lookahead_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
  gj_lookahead_kernel<<<batch, GJLA_THREADS, L.total, s>>>(src, src_stride, out, out_stride, n,
                                                           status);
  rci_note_launch();
  return cudaGetLastError();
}

template <typename T, bool SMEM, int R, int TR, int TC, int NT>
cudaError_t launch_gj_reg(cplx<T>* src, int64_t src_stride, cplx<T>* out, int64_t out_stride,
                          int n, int batch, int32_t* status, cudaStream_t s) {
  const GjSmem<T> L(n, NT / 32, SMEM);
  if (L.total > SMEM_LIMIT || n > 32 * R) return cudaErrorInvalidValue;
  if (L.total > 48 * 1024)
    RCI_CUDA_TRY(cudaFuncSetAttribute(gj_regpanel_kernel<T, SMEM, R, TR, TC, NT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
  gj_regpanel_kernel<T, SMEM, R, TR, TC, NT><<<batch, NT, L.total, s>>>(src, src_stride, out,
                                                                        out_stride, n, status);
  rci_note_launch();
  return cudaGetLastError();
}

template <typename T, bool SMEM, int NB, int TR, int TC, int NT>
cudaError_t launch_gj_cfg(cplx<T>* src, int64_t src_stride, cplx<T>* out, int64_t out_stride,
                          int n, int batch, int32_t* status, cudaStream_t s) {
  const GjSmem<T> L(n, NB, SMEM);
  if (L.total > SMEM_LIMIT) return cudaErrorInvalidValue;
  if (L.total > 48 * 1024)
    RCI_CUDA_TRY(cudaFuncSetAttribute(gj_inverse_kernel<T, SMEM, NB, TR, TC, NT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
  gj_inverse_kernel<T, SMEM, NB, TR, TC, NT><<<batch, NT, L.total, s>>>(src, src_stride, out,
                                                                        out_stride, n, status);
  rci_note_launch();
  return cudaGetLastError();
}

// Batched inverses of n x n blocks: FP32 blocks of n <= 160 with the look-ahead kernel
// (block in shared memory, 1024 threads); other FP32 blocks up to 256 and FP64 blocks up to
// 256 with the register-panel kernel (shared memory while the block fits, else in place in
// global memory); larger blocks with gj_inverse_kernel.
template <typename T>
cudaError_t launch_gj_simt(cplx<T>* src, int64_t src_stride, cplx<T>* out, int64_t out_stride,
                           int n, int batch, int32_t* status, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  if (n > 1024) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 4) {
    if (n <= 160 && GjLaSmem(n).total <= SMEM_LIMIT)
      return launch_gj_lookahead(src, src_stride, out, out_stride, n, batch, status, s);
    if (n <= 160 && GjSmem<T>(n, 16, true).total <= SMEM_LIMIT)
      return launch_gj_reg<T, true, 5, 5, 5, 512>(src, src_stride, out, out_stride, n, batch,
                                                  status, s);
    if (n <= 256)
      return launch_gj_reg<T, false, 8, 5, 5, 512>(src, src_stride, out, out_stride, n, batch,
                                                   status, s);
    return launch_gj_cfg<T, false, 16, 5, 5, 512>(src, src_stride, out, out_stride, n, batch,
                                                  status, s);
  } else {
    if (n <= 160 && GjSmem<T>(n, 8, true).total <= SMEM_LIMIT)
      return launch_gj_reg<T, true, 5, 5, 5, 256>(src, src_stride, out, out_stride, n, batch,
                                                  status, s);
    if (n <= 256)
      return launch_gj_reg<T, false, 8, 5, 5, 256>(src, src_stride, out, out_stride, n, batch,
                                                   status, s);
    if (GjSmem<T>(n, 16, false).total <= SMEM_LIMIT)
      return launch_gj_cfg<T, false, 16, 5, 5, 256>(src, src_stride, out, out_stride, n, batch,
                                                    status, s);
    return launch_gj_cfg<T, false, 8, 5, 5, 256>(src, src_stride, out, out_stride, n, batch,
                                                 status, s);
  }
}

// Batched inverses: FP32 blocks of n <= 160 on the tensor cores (tc_gj.cu: blocked
// Gauss-Jordan with tcgen05 panel updates, block in tensor memory); everything else with the
// SIMT kernels above.
// Largest |re|, |im| over `batch` n x n blocks (stride in elements) into *maxabs (float bits,
// atomicMax), for the growth estimate of the SIMT paths (the tensor-core kernel records it
// while it reads its blocks).
template <typename T>
__global__ void block_maxabs_kernel(const cplx<T>* __restrict__ a, int64_t stride, int64_t nn,
                                    int batch, uint32_t* maxabs) {
  float m = 0.f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn * batch;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t z = e / nn;
    const cplx<T> v = a[z * stride + (e - z * nn)];
    m = fmaxf(m, (float)fmax(fabs(v.x), fabs(v.y)));
  }
  const uint32_t wm = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
  if ((threadIdx.x & 31) == 0) atomicMax(maxabs, wm);
}

template <typename T>
cudaError_t launch_gj(cplx<T>* src, int64_t src_stride, cplx<T>* out, int64_t out_stride, int n,
                      int batch, int32_t* status, cudaStream_t s, uint32_t* maxabs = nullptr,
                      bool tc = true) {
  if (batch <= 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    if (tc && n <= 160)
      return launch_tc_gj(src, src_stride, out, out_stride, n, batch, status, s, maxabs);
  }
  if (maxabs) {
    const int64_t nn = (int64_t)n * n;
    const int64_t tot = nn * batch;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(tot, 256), 4 * 152);
    block_maxabs_kernel<T><<<grid, 256, 0, s>>>(src, src_stride, nn, batch, maxabs);
    rci_note_launch();
    RCI_CUDA_TRY(cudaGetLastError());
  }
  return launch_gj_simt<T>(src, src_stride, out, out_stride, n, batch, status, s);
}

// Largest |re|, |im| of the operator's coefficients (diagonal and couplings)
__global__ void coeff_maxabs_kernel(const double2* __restrict__ dg, const double2* __restrict__ cx,
                                    const double2* __restrict__ cy, int64_t N, uint32_t* maxabs) {
  float m = 0.f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = dg[e], b = cx[e], c = cy[e];
    const double v = fmax(fmax(fmax(fabs(a.x), fabs(a.y)), fmax(fabs(b.x), fabs(b.y))),
                          fmax(fabs(c.x), fabs(c.y)));
    m = fmaxf(m, (float)v);
  }
  const uint32_t wm = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
  if ((threadIdx.x & 31) == 0) atomicMax(maxabs, wm);
}

// ===================================================================== batched GEMM
// C[z] = alpha op(A[z]) op(B[z]) + beta C0[z]   (row-major, complex, op = N or T,
// no conjugation), z = blockIdx.z.  16 x 16 threads, each TM x TN outputs (strided
// by 16 so shared-memory reads are conflict-free), K tiles of 16.
template <typename T>
struct GemmArgs {
  int M, N, K;
  const cplx<T>* A;
  int64_t lda, sA;
  const cplx<T>* B;
  int64_t ldb, sB;
  cplx<T>* C;
  int64_t ldc, sC;
  const cplx<T>* C0;
  int64_t ldc0, sC0;
  cplx<T> alpha, beta;
};

template <typename T, int TM, int TN, bool TA, bool TB>
__global__ void __launch_bounds__(256) cgemm_kernel(GemmArgs<T> p) {
  constexpr int BM = 16 * TM, BN = 16 * TN, BK = 16;
  __shared__ cplx<T> As[BK][BM];
  __shared__ cplx<T> Bs[BK][BN];
  const int64_t z = blockIdx.z;
  const cplx<T>* A = p.A + z * p.sA;
  const cplx<T>* B = p.B + z * p.sB;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  cplx<T> acc[TM][TN];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) acc[r][c] = czero<T>();
  for (int k0 = 0; k0 < p.K; k0 += BK) {
#pragma unroll
    for (int e = tid; e < BM * BK; e += 256) {
      int i, kk;
      if (!TA) {
        i = e / BK;
        kk = e - i * BK;
      } else {
        kk = e / BM;
        i = e - kk * BM;
      }
      int gi = i0 + i, gk = k0 + kk;
      cplx<T> v = czero<T>();
      if (gi < p.M && gk < p.K) v = TA ? A[(int64_t)gk * p.lda + gi] : A[(int64_t)gi * p.lda + gk];
      As[kk][i] = v;
    }
#pragma unroll
    for (int e = tid; e < BK * BN; e += 256) {
      int j, kk;
      if (!TB) {
        kk = e / BN;
        j = e - kk * BN;
      } else {
        j = e / BK;
        kk = e - j * BK;
      }
      int gj = j0 + j, gk = k0 + kk;
      cplx<T> v = czero<T>();
      if (gj < p.N && gk < p.K) v = TB ? B[(int64_t)gj * p.ldb + gk] : B[(int64_t)gk * p.ldb + gj];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cplx<T> av[TM], bv[TN];
#pragma unroll
      for (int r = 0; r < TM; ++r) av[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < TN; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = cfma(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }
  cplx<T>* C = p.C + z * p.sC;
  const cplx<T>* C0 = p.C0 ? p.C0 + z * p.sC0 : nullptr;
#pragma unroll
  for (int r = 0; r < TM; ++r) {
    int gi = i0 + ty + 16 * r;
    if (gi >= p.M) continue;
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      int gj = j0 + tx + 16 * c;
      if (gj >= p.N) continue;
      cplx<T> v = p.alpha * acc[r][c];
      if (C0) v = cfma(p.beta, C0[(int64_t)gi * p.ldc0 + gj], v);
      C[(int64_t)gi * p.ldc + gj] = v;
    }
  }
}

inline int pick_tile(int d) {
  if (d % 80 == 0) return 5;
  if (d % 64 == 0) return 4;
  if (d % 48 == 0) return 3;
  if (d <= 48) return 3;
  return 4;
}

template <typename T, int TM, int TN>
cudaError_t gemm_tn(const GemmArgs<T>& a, bool ta, bool tb, int batch, cudaStream_t s) {
  dim3 grd((unsigned)ceil_div(a.N, 16 * TN), (unsigned)ceil_div(a.M, 16 * TM), (unsigned)batch);
  if (!ta && !tb) cgemm_kernel<T, TM, TN, false, false><<<grd, 256, 0, s>>>(a);
  else if (!ta && tb) cgemm_kernel<T, TM, TN, false, true><<<grd, 256, 0, s>>>(a);
  else if (ta && !tb) cgemm_kernel<T, TM, TN, true, false><<<grd, 256, 0, s>>>(a);
  else return cudaErrorInvalidValue;
  rci_note_launch();
  return cudaGetLastError();
}

template <typename T, int TM>
cudaError_t gemm_m(const GemmArgs<T>& a, bool ta, bool tb, int batch, cudaStream_t s) {
  switch (pick_tile(a.N)) {
    case 3: return gemm_tn<T, TM, 3>(a, ta, tb, batch, s);
    case 5: return gemm_tn<T, TM, 5>(a, ta, tb, batch, s);
    default: return gemm_tn<T, TM, 4>(a, ta, tb, batch, s);
  }
}

// Batched GEMM with element strides between the batch members.
template <typename T>
cudaError_t gemm(int M, int N, int K, bool ta, bool tb, cplx<T> alpha, const cplx<T>* A,
                 int64_t lda, int64_t sA, const cplx<T>* B, int64_t ldb, int64_t sB, cplx<T> beta,
                 const cplx<T>* C0, int64_t ldc0, int64_t sC0, cplx<T>* C, int64_t ldc,
                 int64_t sC, int batch, cudaStream_t s, Profiler* prof = nullptr,
                 int fam = PF_GEMM, int32_t* status = nullptr) {
  if (batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  ProfScope ps(prof, fam, s, 8.0 * M * N * K * (double)batch,
               (double)sizeof(cplx<T>) * batch * ((double)M * K + (double)K * N + (double)M * N), 1);
  GemmArgs<T> a{M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, C0, ldc0, sC0, alpha, beta};
  // small batches (the last reduction levels) leave most SMs idle with large tiles and
  // are latency-bound: use 32 x 32 output tiles there
  const int64_t big_tiles = (int64_t)batch * ceil_div(M, 80) * ceil_div(N, 80);
  // FP32 products run on the tensor cores (3xTF32): the TMA-fed kernel at any batch where it
  // applies (its 64-row tiles keep even one product on several SMs, and a tile takes a few
  // microseconds); the register-staged kernels where enough tiles fill the GPU
  if constexpr (sizeof(T) == 4) {
    if (status && alpha.y == 0.f && beta.y == 0.f) {
      const cudaError_t e = launch_tc_cgemm_tma(M, N, K, ta, tb, alpha.x, A, lda, sA, B, ldb, sB,
                                                beta.x, C0, ldc0, sC0, C, ldc, sC, batch, status,
                                                tc_wait_limit(), s);
      if (e != cudaErrorNotSupported) return e;
    }
    const int64_t tc_tiles = (int64_t)batch * ceil_div(M, 128) * ceil_div(N, 80);
    if (status && tc_tiles >= 152)
      return launch_tc_cgemm(M, N, K, ta, tb, alpha, A, lda, sA, B, ldb, sB, beta, C0, ldc0, sC0,
                             C, ldc, sC, batch, status, s, 1);
  }
  if (big_tiles < 2 * 152) return gemm_tn<T, 2, 2>(a, ta, tb, batch, s);
  switch (pick_tile(M)) {
    case 3: return gemm_m<T, 3>(a, ta, tb, batch, s);
    case 5: return gemm_m<T, 5>(a, ta, tb, batch, s);
    default: return gemm_m<T, 4>(a, ta, tb, batch, s);
  }
}

// ===================================================================== solve kernels
// Level 0 forward: t0[k] = T_{2k+1}^{-1} b[2k+1] (one thread per (k, q)).
template <typename T>
__global__ void fwd0_kernel(const cplx<T>* __restrict__ b, cplx<T>* __restrict__ t0, int ny,
                            int m0, int nrhs, const cplx<T>* tdl, const cplx<T>* tdinv,
                            const cplx<T>* tdu, const cplx<T>* tdu2, const uint8_t* tpiv) {
  int64_t tt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tt >= (int64_t)m0 * nrhs) return;
  int k = (int)(tt / nrhs), q = (int)(tt - (int64_t)k * nrhs);
  int64_t fb = (int64_t)k * ny;
  TriRow<T> f{tdl + fb, tdinv + fb, tdu + fb, tdu2 + fb, tpiv + fb};
  const cplx<T>* br = b + (2 * (int64_t)k + 1) * ny * nrhs + q;
  cplx<T>* tr = t0 + (int64_t)k * ny * nrhs + q;
  tri_forward<T>(f, ny, [&](int j) { return br[(int64_t)j * nrhs]; },
                 [&](int j, cplx<T> y) { tr[(int64_t)j * nrhs] = y; });
  tri_backward<T>(f, ny, [&](int j) { return tr[(int64_t)j * nrhs]; },
                  [&](int j, cplx<T> g) { tr[(int64_t)j * nrhs] = g; });
}

// Level 0 kept rows: B1[k] = b[2k] - cx[2k-1] o t0[k-1] - cx[2k] o t0[k].
template <typename T>
__global__ void keep0_kernel(const cplx<T>* __restrict__ b, const cplx<T>* __restrict__ t0,
                             const double2* __restrict__ cx, cplx<T>* __restrict__ B1, int nx,
                             int ny, int n1, int nrhs) {
  int64_t row = (int64_t)ny * nrhs;
  int64_t tt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tt >= (int64_t)n1 * row) return;
  int64_t k = tt / row, r = tt - k * row;
  int j = (int)(r / nrhs);
  cplx<T> v = b[2 * k * row + r];
  if (k >= 1) v = cfms(ccast<T>(cx[(2 * k - 1) * ny + j]), t0[(k - 1) * row + r], v);
  if (2 * k + 1 < nx) v = cfms(ccast<T>(cx[(2 * k) * ny + j]), t0[k * row + r], v);
  B1[tt] = v;
}

// Level 0 back substitution: x[2k] = x1[k];
// x[2k+1] = T^{-1}(b[2k+1] - cx[2k] o x1[k] - cx[2k+1] o x1[k+1]).
template <typename T>
__global__ void bwd0_kernel(const cplx<T>* b, const cplx<T>* __restrict__ x1,
                            const double2* __restrict__ cx, cplx<T>* x, int nx, int ny, int n1,
                            int nrhs, const cplx<T>* tdl, const cplx<T>* tdinv, const cplx<T>* tdu,
                            const cplx<T>* tdu2, const uint8_t* tpiv) {
  int64_t tt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tt >= (int64_t)n1 * nrhs) return;
  int k = (int)(tt / nrhs), q = (int)(tt - (int64_t)k * nrhs);
  int64_t row = (int64_t)ny * nrhs;
  const cplx<T>* xa = x1 + (int64_t)k * row + q;
  cplx<T>* xe = x + 2 * (int64_t)k * row + q;
  for (int j = 0; j < ny; ++j) xe[(int64_t)j * nrhs] = xa[(int64_t)j * nrhs];
  int64_t r = 2 * (int64_t)k + 1;
  if (r >= nx) return;
  const bool has_b = r + 1 < nx;
  const cplx<T>* xb = x1 + (int64_t)(k + 1) * row + q;
  const cplx<T>* br = b + r * row + q;
  cplx<T>* xr = x + r * row + q;
  const double2* cl = cx + (r - 1) * ny;
  const double2* cr = cx + r * ny;
  int64_t fb = (int64_t)k * ny;
  TriRow<T> f{tdl + fb, tdinv + fb, tdu + fb, tdu2 + fb, tpiv + fb};
  auto rhs = [&](int j) {
    cplx<T> v = cfms(ccast<T>(cl[j]), xa[(int64_t)j * nrhs], br[(int64_t)j * nrhs]);
    if (has_b) v = cfms(ccast<T>(cr[j]), xb[(int64_t)j * nrhs], v);
    return v;
  };
  tri_forward<T>(f, ny, rhs, [&](int j, cplx<T> y) { xr[(int64_t)j * nrhs] = y; });
  tri_backward<T>(f, ny, [&](int j) { return xr[(int64_t)j * nrhs]; },
                  [&](int j, cplx<T> g) { xr[(int64_t)j * nrhs] = g; });
}

// Kept rows of a dense level: Bn[k] = B[2k] - Q[k-1] - P[k].
template <typename T>
__global__ void keep_kernel(const cplx<T>* __restrict__ B, const cplx<T>* __restrict__ P,
                            const cplx<T>* __restrict__ Q, cplx<T>* __restrict__ Bn, int m, int nk,
                            int64_t row) {
  int64_t tt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tt >= (int64_t)nk * row) return;
  int64_t k = tt / row, r = tt - k * row;
  cplx<T> v = B[2 * k * row + r];
  if (k >= 1) v = v - Q[(k - 1) * row + r];
  if (k < m) v = v - P[k * row + r];
  Bn[tt] = v;
}

// x_l[2k] = x_up[k] for every kept row.
template <typename T>
__global__ void copy_kept_kernel(const cplx<T>* __restrict__ xup, cplx<T>* __restrict__ xl, int nk,
                                 int64_t row) {
  int64_t tt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tt >= (int64_t)nk * row) return;
  int64_t k = tt / row, r = tt - k * row;
  xl[2 * k * row + r] = xup[tt];
}

// sum of a complex value over the 32 lanes of a warp (every lane gets the sum)
template <typename T>
__device__ __forceinline__ cplx<T> warp_sum(cplx<T> v) {
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  return v;
}

// Level 0 backward, several right-hand sides: x[2k] = x1[k] and the right-hand sides of
// the eliminated rows, tmp[k] = b[2k+1] - cx[2k] o x1[k] - cx[2k+1] o x1[k+1].
template <typename T>
__global__ void bwd0_rhs_kernel(const cplx<T>* b, const cplx<T>* __restrict__ x1,
                                const double2* __restrict__ cx, cplx<T>* x,
                                cplx<T>* __restrict__ tmp, int nx, int ny, int n1, int nrhs) {
  const int64_t row = (int64_t)ny * nrhs;
  const int64_t tt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tt >= (int64_t)n1 * row) return;
  const int64_t k = tt / row, e = tt - k * row;
  const int j = (int)(e / nrhs);
  const int64_t r = 2 * k + 1;
  const cplx<T> xa = x1[tt];
  if (r < nx) {
    cplx<T> v = cfms(ccast<T>(cx[(r - 1) * ny + j]), xa, b[r * row + e]);
    if (r + 1 < nx) v = cfms(ccast<T>(cx[r * ny + j]), x1[(k + 1) * row + e], v);
    tmp[k * row + e] = v;
  }
  x[2 * k * row + e] = xa;
}

// ----- single right-hand side, chunked: a block per (block row k, chunk of RC rows or
// columns), so that even the last reduction levels spread over many SMs, and every lane
// issues all of its 16-byte loads before it reduces.
constexpr int RC = 32;
constexpr int CH_THREADS = 256, CH_WARPS = CH_THREADS / 32;

template <typename T> struct vec16;
template <> struct vec16<float> { using type = float4; static constexpr int per = 2; };
template <> struct vec16<double> { using type = double2; static constexpr int per = 1; };

template <typename T>
__device__ __forceinline__ cplx<T> dot_vec(const typename vec16<T>::type& v, const cplx<T>* x,
                                           int c, cplx<T> acc) {
  if constexpr (sizeof(T) == 4) {
    acc = cfma(mkc(v.x, v.y), x[c], acc);
    return cfma(mkc(v.z, v.w), x[c + 1], acc);
  } else {
    return cfma(v, x[c], acc);
  }
}

// out[r] (= sub[r] -) M[r, :] x  for the RC rows r0 .. r0+RC-1 (x in shared memory).
// Warp w handles rows r0 + w + CH_WARPS i; SMAX 16-byte vectors per lane and row.
template <typename T, int SMAX>
__device__ __forceinline__ void rows_mv(const cplx<T>* __restrict__ M, const cplx<T>* x, int ny,
                                        int r0, cplx<T>* out, const cplx<T>* sub) {
  using V = typename vec16<T>::type;
  constexpr int PER = vec16<T>::per;
  constexpr int RPW = RC / CH_WARPS;  // rows per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nv = ny / PER;            // ny is a multiple of PER (checked by the launcher)
  V v[RPW][SMAX];
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = r0 + warp + CH_WARPS * i;
    const V* Mr = reinterpret_cast<const V*>(M + (int64_t)r * ny);
#pragma unroll
    for (int s = 0; s < SMAX; ++s) {
      const int q = lane + 32 * s;
      if (r < ny && q < nv) v[i][s] = __ldg(Mr + q);
    }
  }
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = r0 + warp + CH_WARPS * i;
    cplx<T> acc = czero<T>();
#pragma unroll
    for (int s = 0; s < SMAX; ++s) {
      const int q = lane + 32 * s;
      if (r < ny && q < nv) acc = dot_vec<T>(v[i][s], x, PER * q, acc);
    }
    acc = warp_sum<T>(acc);
    if (lane == 0 && r < ny) out[r] = sub ? sub[r] - acc : acc;
  }
}

// rows_mv split in two: the row loads (no dependence on x) and the products, so that a
// block can issue its loads before it waits for the vector it multiplies.
template <typename T, int SMAX>
struct Rows1 {
  typename vec16<T>::type v[RC / CH_WARPS][SMAX];
};

template <typename T, int SMAX>
__device__ __forceinline__ void rows_load1(Rows1<T, SMAX>& R, const cplx<T>* __restrict__ M, int ny,
                                           int r0) {
  using V = typename vec16<T>::type;
  constexpr int PER = vec16<T>::per;
  constexpr int RPW = RC / CH_WARPS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nv = ny / PER;
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = r0 + warp + CH_WARPS * i;
    const V* Mr = reinterpret_cast<const V*>(M + (int64_t)r * ny);
#pragma unroll
    for (int s = 0; s < SMAX; ++s) {
      const int q = lane + 32 * s;
      if (r < ny && q < nv) R.v[i][s] = __ldg(Mr + q);
    }
  }
}

template <typename T, int SMAX>
__device__ __forceinline__ void rows_dot1(const Rows1<T, SMAX>& R, const cplx<T>* x, int ny, int r0,
                                          cplx<T>* out) {
  constexpr int PER = vec16<T>::per;
  constexpr int RPW = RC / CH_WARPS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nv = ny / PER;
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = r0 + warp + CH_WARPS * i;
    cplx<T> acc = czero<T>();
#pragma unroll
    for (int s = 0; s < SMAX; ++s) {
      const int q = lane + 32 * s;
      if (r < ny && q < nv) acc = dot_vec<T>(R.v[i][s], x, PER * q, acc);
    }
    acc = warp_sum<T>(acc);
    if (lane == 0 && r < ny) out[r] = acc;
  }
}

// out[r] = sub[r] - M1[r, :] x1 - M2[r, :] x2 for the RC rows r0 .. r0+RC-1: both
// matrices' row vectors are loaded before any product, so a block streams its 2 x RC rows
// in one memory phase (the sums are formed in the order of two rows_mv calls).
template <typename T, int SMAX>
struct Rows2 {  // this thread's 16-byte vectors of the RPW rows of two matrices
  typename vec16<T>::type v1[RC / CH_WARPS][SMAX], v2[RC / CH_WARPS][SMAX];
};

// Issue the loads of rows r0 + warp + CH_WARPS i of M1 and M2 (no dependence on x).
template <typename T, int SMAX>
__device__ __forceinline__ void rows_load2(Rows2<T, SMAX>& R, const cplx<T>* __restrict__ M1,
                                           const cplx<T>* __restrict__ M2, int ny, int r0) {
  using V = typename vec16<T>::type;
  constexpr int PER = vec16<T>::per;
  constexpr int RPW = RC / CH_WARPS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nv = ny / PER;
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = r0 + warp + CH_WARPS * i;
    const V* A = reinterpret_cast<const V*>(M1 + (int64_t)r * ny);
    const V* B = reinterpret_cast<const V*>(M2 + (int64_t)r * ny);
#pragma unroll
    for (int s = 0; s < SMAX; ++s) {
      const int q = lane + 32 * s;
      if (r < ny && q < nv) {
        R.v1[i][s] = __ldg(A + q);
        R.v2[i][s] = __ldg(B + q);
      }
    }
  }
}

// out[r] = (sub[r] - M1[r] . x1) - M2[r] . x2 for the rows loaded by rows_load2 (x1, x2 in
// shared memory).
template <typename T, int SMAX>
__device__ __forceinline__ void rows_dot2(const Rows2<T, SMAX>& R, const cplx<T>* x1,
                                          const cplx<T>* x2, int ny, int r0, cplx<T>* out,
                                          const cplx<T>* sub) {
  constexpr int PER = vec16<T>::per;
  constexpr int RPW = RC / CH_WARPS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nv = ny / PER;
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = r0 + warp + CH_WARPS * i;
    cplx<T> a1 = czero<T>(), a2 = czero<T>();
#pragma unroll
    for (int s = 0; s < SMAX; ++s) {
      const int q = lane + 32 * s;
      if (r < ny && q < nv) {
        a1 = dot_vec<T>(R.v1[i][s], x1, PER * q, a1);
        a2 = dot_vec<T>(R.v2[i][s], x2, PER * q, a2);
      }
    }
    a1 = warp_sum<T>(a1);
    a2 = warp_sum<T>(a2);
    if (lane == 0 && r < ny) out[r] = (sub[r] - a1) - a2;
  }
}

// out[c] = sum_a M[a][c] x[a] for the RC columns c0 .. c0+RC-1 (x in shared memory);
// lanes own columns, warps stride over rows, partial sums reduced through red[CH_WARPS][RC].
template <typename T>
__device__ __forceinline__ void cols_mvT(const cplx<T>* __restrict__ M, const cplx<T>* x, int ny,
                                         int c0, cplx<T>* red, cplx<T>* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = c0 + lane;
  cplx<T> acc = czero<T>();
  constexpr int U = 5;
  for (int a0 = warp; a0 < ny; a0 += CH_WARPS * U) {
    cplx<T> m[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int a = a0 + CH_WARPS * u;
      m[u] = (a < ny && c < ny) ? __ldg(M + (int64_t)a * ny + c) : czero<T>();
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int a = a0 + CH_WARPS * u;
      if (a < ny) acc = cfma(m[u], x[a], acc);
    }
  }
  red[warp * RC + lane] = acc;
  __syncthreads();
  if (warp == 0) {
    cplx<T> s = czero<T>();
#pragma unroll
    for (int w = 0; w < CH_WARPS; ++w) s = s + red[w * RC + lane];
    if (c < ny) out[c] = s;
  }
  __syncthreads();
}

// outP[c] = sum_a X[a][c] x[a] and, if Y, outQ[c] = sum_a Y[a][c] x[a], for the RC columns
// c0 .. c0+RC-1, the loads of both matrices in one loop (the sums are formed in the order of
// two cols_mvT calls); red holds 2 x CH_WARPS x RC entries.
template <typename T>
__device__ __forceinline__ void cols_mvT2(const cplx<T>* __restrict__ X,
                                          const cplx<T>* __restrict__ Y, const cplx<T>* x, int ny,
                                          int c0, cplx<T>* red, cplx<T>* outP, cplx<T>* outQ) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = c0 + lane;
  cplx<T> ap = czero<T>(), aq = czero<T>();
  constexpr int U = 5;
  for (int a0 = warp; a0 < ny; a0 += CH_WARPS * U) {
    cplx<T> mx[U], my[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int a = a0 + CH_WARPS * u;
      const bool v = a < ny && c < ny;
      mx[u] = v ? __ldg(X + (int64_t)a * ny + c) : czero<T>();
      my[u] = (v && Y) ? __ldg(Y + (int64_t)a * ny + c) : czero<T>();
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int a = a0 + CH_WARPS * u;
      if (a < ny) {
        ap = cfma(mx[u], x[a], ap);
        aq = cfma(my[u], x[a], aq);
      }
    }
  }
  red[warp * RC + lane] = ap;
  red[(CH_WARPS + warp) * RC + lane] = aq;
  __syncthreads();
  if (warp == 0) {
    cplx<T> sp = czero<T>(), sq = czero<T>();
#pragma unroll
    for (int w = 0; w < CH_WARPS; ++w) {
      sp = sp + red[w * RC + lane];
      sq = sq + red[(CH_WARPS + w) * RC + lane];
    }
    if (c < ny) {
      outP[c] = sp;
      if (Y) outQ[c] = sq;
    }
  }
  __syncthreads();
}

// Dense level, forward: t_k = Dinv_k b_{2k+1} (rows of chunk), P_k = X_k^T b_{2k+1},
// Q_k = Y_k^T b_{2k+1} (columns of chunk).  Grid (m, ceil(ny / RC)).
template <typename T, int SMAX>
__global__ void __launch_bounds__(CH_THREADS)
fwd_chunk_kernel(const cplx<T>* __restrict__ Dinv, const cplx<T>* __restrict__ X,
                 const cplx<T>* __restrict__ Y, const cplx<T>* __restrict__ B,
                 cplx<T>* __restrict__ t, cplx<T>* __restrict__ P, cplx<T>* __restrict__ Q, int n,
                 int ny) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<T>* bs = reinterpret_cast<cplx<T>*>(sm_raw);
  cplx<T>* red = bs + ny;
  const int64_t k = blockIdx.x;
  const int c0 = blockIdx.y * RC;
  const int64_t nn = (int64_t)ny * ny;
  // the Dinv rows of the chunk are loaded before b (rows up to 192 columns in FP32)
  constexpr bool early = sizeof(T) == 4 && SMAX <= 3;
  Rows1<T, early ? SMAX : 1> R;
  if constexpr (early) rows_load1<T, SMAX>(R, Dinv + k * nn, ny, c0);
  for (int c = threadIdx.x; c < ny; c += CH_THREADS) bs[c] = B[(2 * k + 1) * ny + c];
  __syncthreads();
  if constexpr (early) rows_dot1<T, SMAX>(R, bs, ny, c0, t + k * ny);
  else rows_mv<T, SMAX>(Dinv + k * nn, bs, ny, c0, t + k * ny, nullptr);
  // X^T b and Y^T b on the chunk columns, both matrices streamed together
  cols_mvT2<T>(X + k * nn, 2 * k + 2 < n ? Y + k * nn : nullptr, bs, ny, c0, red, P + k * ny,
               Q + k * ny);
}

// Dense level, backward: x_l[2k] = x_up[k];
// x_l[2k+1] = t_k - X_k x_up[k] - Y_k x_up[k+1] (rows of chunk).  Grid (nk, ceil(ny / RC)).
template <typename T, int SMAX>
__global__ void __launch_bounds__(CH_THREADS)
bwd_chunk_kernel(const cplx<T>* __restrict__ X, const cplx<T>* __restrict__ Y,
                 const cplx<T>* __restrict__ t, const cplx<T>* __restrict__ xup,
                 cplx<T>* __restrict__ xl, int n, int m, int ny) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<T>* xa = reinterpret_cast<cplx<T>*>(sm_raw);
  cplx<T>* xb = xa + ny;
  cplx<T>* tmp = xb + ny;
  const int64_t k = blockIdx.x;
  const int c0 = blockIdx.y * RC;
  const int64_t nn = (int64_t)ny * ny;
  const bool has_b = 2 * k + 2 < n;
  // x = (t - X xa) - Y xb on the chunk rows; X and Y rows streamed together where the
  // register tiles of both fit (FP32 rows up to 192 columns), their loads issued before
  // the vectors they multiply are read, else one after the other
  // (early loads for rows up to 192 columns, where the register tiles keep two CTAs per SM)
  constexpr bool fuse = sizeof(T) == 4 && SMAX <= 6;
  constexpr bool early = fuse && SMAX <= 3;
  const bool fused = fuse && has_b && k < m;
  Rows2<T, fuse ? SMAX : 1> R;
  if constexpr (early) {
    if (fused) rows_load2<T, SMAX>(R, X + k * nn, Y + k * nn, ny, c0);
  }
  for (int c = threadIdx.x; c < ny; c += CH_THREADS) {
    xa[c] = xup[k * ny + c];
    xb[c] = has_b ? xup[(k + 1) * ny + c] : czero<T>();
  }
  for (int c = c0 + threadIdx.x; c < c0 + RC && c < ny; c += CH_THREADS)
    xl[2 * k * ny + c] = xup[k * ny + c];
  __syncthreads();
  if (k >= m) return;
  if (fused) {
    if constexpr (fuse) {
      if constexpr (!early) rows_load2<T, SMAX>(R, X + k * nn, Y + k * nn, ny, c0);
      rows_dot2<T, SMAX>(R, xa, xb, ny, c0, xl + (2 * k + 1) * ny, t + k * ny);
    }
  } else if (has_b) {
    rows_mv<T, SMAX>(X + k * nn, xa, ny, c0, tmp, t + k * ny);
    __syncthreads();
    rows_mv<T, SMAX>(Y + k * nn, xb, ny, c0, xl + (2 * k + 1) * ny, tmp);
  } else {
    rows_mv<T, SMAX>(X + k * nn, xa, ny, c0, tmp, t + k * ny);
    __syncthreads();
    for (int c = c0 + threadIdx.x; c < c0 + RC && c < ny; c += CH_THREADS)
      xl[(2 * k + 1) * ny + c] = tmp[c];
  }
}

// y_k = M_k v_k for stored inverses (level 0 forward, the last single row): the vector
// is row vrow of V (stride ny).  Grid (batch, ceil(ny / RC)).
template <typename T, int SMAX>
__global__ void __launch_bounds__(CH_THREADS)
mv_chunk_kernel(const cplx<T>* __restrict__ M, const cplx<T>* __restrict__ V, int64_t v_stride,
                int64_t v_off, cplx<T>* __restrict__ y, int ny) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<T>* vs = reinterpret_cast<cplx<T>*>(sm_raw);
  const int64_t k = blockIdx.x;
  for (int c = threadIdx.x; c < ny; c += CH_THREADS) vs[c] = V[k * v_stride + v_off + c];
  __syncthreads();
  rows_mv<T, SMAX>(M + k * (int64_t)ny * ny, vs, ny, blockIdx.y * RC, y + k * ny, nullptr);
}

// Row r of a level's right-hand side formed from the level before it (Bp, its P, Q and
// mp eliminated rows): b[r] = Bp[2r] - Qp[r-1] - Pp[r], the Q term for r >= 1 and the P term
// for r < mp, in keep_kernel's order (so the values are the ones keep_kernel would store).
template <typename T>
__device__ __forceinline__ cplx<T> kept_row(const cplx<T>* __restrict__ Bp,
                                            const cplx<T>* __restrict__ Pp,
                                            const cplx<T>* __restrict__ Qp, int mp, int64_t r,
                                            int c, int ny) {
  cplx<T> v = Bp[2 * r * ny + c];
  if (r >= 1) v = v - Qp[(r - 1) * ny + c];
  if (r < mp) v = v - Pp[r * ny + c];
  return v;
}

// Dense level l >= 2, forward, with the kept-row update of level l - 1 fused in: block
// (k, chunk) forms the odd row 2k + 1 of this level's right-hand side whole in shared memory
// and then t_k, P_k, Q_k on its chunk as fwd_chunk_kernel does; it also writes the even row
// 2k on its chunk to Bn, from which the next level forms its rows.  Grid (ceil(n / 2),
// ceil(ny / RC)): for odd n the last block row k = n / 2 has its even row only.
template <typename T, int SMAX>
__global__ void __launch_bounds__(CH_THREADS)
fwd_keep_chunk_kernel(const cplx<T>* __restrict__ Dinv, const cplx<T>* __restrict__ X,
                      const cplx<T>* __restrict__ Y, const cplx<T>* __restrict__ Bp,
                      const cplx<T>* __restrict__ Pp, const cplx<T>* __restrict__ Qp, int mp,
                      cplx<T>* __restrict__ Bn, cplx<T>* __restrict__ t, cplx<T>* __restrict__ P,
                      cplx<T>* __restrict__ Q, int n, int ny) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<T>* bs = reinterpret_cast<cplx<T>*>(sm_raw);
  cplx<T>* red = bs + ny;
  const int64_t k = blockIdx.x;
  const int c0 = blockIdx.y * RC;
  const int64_t nn = (int64_t)ny * ny;
  for (int c = c0 + threadIdx.x; c < c0 + RC && c < ny; c += CH_THREADS)
    Bn[2 * k * ny + c] = kept_row<T>(Bp, Pp, Qp, mp, 2 * k, c, ny);
  if (2 * k + 1 >= n) return;  // (uniform over the block)
  constexpr bool early = sizeof(T) == 4 && SMAX <= 3;
  Rows1<T, early ? SMAX : 1> R;
  if constexpr (early) rows_load1<T, SMAX>(R, Dinv + k * nn, ny, c0);
  for (int c = threadIdx.x; c < ny; c += CH_THREADS)
    bs[c] = kept_row<T>(Bp, Pp, Qp, mp, 2 * k + 1, c, ny);
  __syncthreads();
  if constexpr (early) rows_dot1<T, SMAX>(R, bs, ny, c0, t + k * ny);
  else rows_mv<T, SMAX>(Dinv + k * nn, bs, ny, c0, t + k * ny, nullptr);
  cols_mvT2<T>(X + k * nn, 2 * k + 2 < n ? Y + k * nn : nullptr, bs, ny, c0, red, P + k * ny,
               Q + k * ny);
}

// The single last row with the kept-row update of the level before it fused in:
// y = M b[0], b[0] = Bp[0] - Pp[0] (mp > 0).  Grid (1, ceil(ny / RC)).
template <typename T, int SMAX>
__global__ void __launch_bounds__(CH_THREADS)
mv_keep_chunk_kernel(const cplx<T>* __restrict__ M, const cplx<T>* __restrict__ Bp,
                     const cplx<T>* __restrict__ Pp, const cplx<T>* __restrict__ Qp, int mp,
                     cplx<T>* __restrict__ y, int ny) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<T>* vs = reinterpret_cast<cplx<T>*>(sm_raw);
  for (int c = threadIdx.x; c < ny; c += CH_THREADS) vs[c] = kept_row<T>(Bp, Pp, Qp, mp, 0, c, ny);
  __syncthreads();
  rows_mv<T, SMAX>(M, vs, ny, blockIdx.y * RC, y, nullptr);
}

// ----- single right-hand side, level 0 by the pivoted tridiagonal factors (5 ny values per
// eliminated row instead of the dense ny x ny inverse): one warp per eliminated row k stages
// the row's factors and right-hand side in shared memory, lane 0 runs the forward and
// backward sweeps, the warp writes the result.
//   FWD: t0[k] = T_{2k+1}^{-1} b[2k+1]
//   BWD: x[2k] = x1[k];  x[2k+1] = T_{2k+1}^{-1} (b[2k+1] - cx[2k] o x1[k] - cx[2k+1] o x1[k+1])
constexpr int TRS_WARPS = 4;

template <typename T>
__host__ __device__ size_t trs_smem_per_warp(int ny) {
  return ((size_t)5 * ny * sizeof(cplx<T>) + (size_t)ny + 15) & ~(size_t)15;
}

template <typename T, bool BWD>
__global__ void __launch_bounds__(32 * TRS_WARPS)
tri_rows_solve_kernel(const cplx<T>* __restrict__ tdl, const cplx<T>* __restrict__ tdinv,
                      const cplx<T>* __restrict__ tdu, const cplx<T>* __restrict__ tdu2,
                      const uint8_t* __restrict__ tpiv, const cplx<T>* __restrict__ b,
                      const cplx<T>* __restrict__ x1, const double2* __restrict__ cx,
                      cplx<T>* __restrict__ out, int nx, int ny, int rows) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * TRS_WARPS + w;
  if (k >= rows) return;  // whole warp
  cplx<T>* dl = reinterpret_cast<cplx<T>*>(sm_raw + (size_t)w * trs_smem_per_warp<T>(ny));
  cplx<T>* di = dl + ny;
  cplx<T>* du = di + ny;
  cplx<T>* du2 = du + ny;
  cplx<T>* v = du2 + ny;
  uint8_t* pv = reinterpret_cast<uint8_t*>(v + ny);
  const int64_t r = 2 * (int64_t)k + 1;
  const bool has = r < nx;
  if (BWD) {
    for (int j = lane; j < ny; j += 32) out[2 * (int64_t)k * ny + j] = x1[(int64_t)k * ny + j];
  }
  if (!has) return;
  const int64_t fb = (int64_t)k * ny;
  for (int j = lane; j < ny; j += 32) {
    dl[j] = tdl[fb + j];
    di[j] = tdinv[fb + j];
    du[j] = tdu[fb + j];
    du2[j] = tdu2[fb + j];
    pv[j] = tpiv[fb + j];
    cplx<T> rv = b[r * ny + j];
    if (BWD) {
      rv = cfms(ccast<T>(cx[(r - 1) * ny + j]), x1[(int64_t)k * ny + j], rv);
      if (r + 1 < nx) rv = cfms(ccast<T>(cx[r * ny + j]), x1[(int64_t)(k + 1) * ny + j], rv);
    }
    v[j] = rv;
  }
  __syncwarp();
  if (lane == 0) {
    TriRow<T> f{dl, di, du, du2, pv};
    tri_forward<T>(f, ny, [&](int j) { return v[j]; }, [&](int j, cplx<T> y) { v[j] = y; });
    tri_backward<T>(f, ny, [&](int j) { return v[j]; }, [&](int j, cplx<T> g) { v[j] = g; });
  }
  __syncwarp();
  cplx<T>* o = BWD ? out + r * ny : out + (int64_t)k * ny;
  for (int j = lane; j < ny; j += 32) o[j] = v[j];
}

}  // namespace

// ===================================================================== handle
struct BcrHandle {
  int prec;
  int nx, ny;
  std::vector<int64_t> n, m;      // rows / eliminated rows per level (index 0 = tridiagonal level)
  std::vector<int64_t> off;       // store offsets (elements) of levels >= 1
  int64_t final_off = 0;
  int Lf = 1;                     // level with a single row
  size_t esz = 0;                 // bytes per complex element
  // factor storage
  void *tdl = nullptr, *tdinv = nullptr, *tdu = nullptr, *tdu2 = nullptr;
  uint8_t* tpiv = nullptr;
  void* G0 = nullptr;             // dense T_r^{-1} of the level-0 eliminated rows (m0 x ny x ny)
  bool g0_valid = false;          // G0 holds the inverses of the current factorisation
  bool simt = false;              // FP32: factor and multi-RHS products on the SIMT pipe
  void* Dw[2] = {nullptr, nullptr};
  void* Lw[2] = {nullptr, nullptr};
  void* store = nullptr;
  int32_t* status = nullptr;
  size_t factor_bytes = 0;
  Profiler* prof = nullptr;
  // solve workspace (grown on demand)
  int ws_nrhs = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  DevMem mem;
};

static void free_ws(BcrHandle* h) {
  h->mem.release(h->ws);
  h->ws = nullptr;
  h->ws_nrhs = 0;
  h->ws_bytes = 0;
}

void bcr_destroy(BcrHandle* h) {
  if (!h) return;
  void* ps[] = {h->tdl, h->tdinv, h->tdu, h->tdu2, h->tpiv, h->G0, h->Dw[0], h->Dw[1],
                h->Lw[0], h->Lw[1], h->store, h->status};
  for (void* p : ps) h->mem.release(p);
  free_ws(h);
  delete h;
}

size_t bcr_bytes(const BcrHandle* h) { return h->factor_bytes + h->ws_bytes; }
void bcr_set_profiler(BcrHandle* h, Profiler* p) { h->prof = p; }
int bcr_precision(const BcrHandle* h) { return h->prec; }
void bcr_set_simt(BcrHandle* h, bool simt) { h->simt = simt && h->prec != RCI_FP64; }
bool bcr_simt(const BcrHandle* h) { return h->simt; }

// The status word handed to gemm<T>: its tensor-core paths run only with one (they record an
// expired bounded wait there), so a handle set to the SIMT pipe passes none.
static int32_t* gemm_status(const BcrHandle* h) { return h->simt ? nullptr : h->status; }

cudaError_t bcr_create(int nx, int ny, int prec, const DevMem* mem, BcrHandle** out, size_t* bytes) {
  *out = nullptr;
  if (nx < 1 || ny < 2 || ny > 1024) return cudaErrorInvalidValue;
  BcrHandle* h = new (std::nothrow) BcrHandle();
  if (!h) return cudaErrorMemoryAllocation;
  if (mem) h->mem = *mem;
  h->prec = prec;
  h->nx = nx;
  h->ny = ny;
  h->esz = prec == RCI_FP64 ? sizeof(double2) : sizeof(float2);
  const int64_t nn = (int64_t)ny * ny;
  h->n.push_back(nx);
  h->m.push_back(nx / 2);
  int64_t cur = (nx + 1) / 2;
  int64_t off = 0;
  h->off.push_back(0);
  int L = 1;
  while (cur > 1) {
    h->n.push_back(cur);
    h->m.push_back(cur / 2);
    h->off.push_back(off);
    off += 3 * (cur / 2) * nn;
    cur = (cur + 1) / 2;
    ++L;
  }
  h->n.push_back(1);
  h->m.push_back(0);
  h->off.push_back(off);
  h->Lf = L;
  h->final_off = off;
  int64_t store_elems = off + nn;
  int64_t m0 = h->m[0], n1 = (nx + 1) / 2;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t b) {
    if (e != cudaSuccess) return;
    e = h->mem.alloc(p, b);
    if (e == cudaSuccess) h->factor_bytes += b;
  };
  size_t m0b = (size_t)std::max<int64_t>(m0, 1) * ny;
  alloc(&h->tdl, m0b * h->esz);
  alloc(&h->tdinv, m0b * h->esz);
  alloc(&h->tdu, m0b * h->esz);
  alloc(&h->tdu2, m0b * h->esz);
  alloc((void**)&h->tpiv, m0b);
  alloc(&h->G0, m0b * ny * h->esz);
  for (int i = 0; i < 2; ++i) {
    alloc(&h->Dw[i], (size_t)n1 * nn * h->esz);
    alloc(&h->Lw[i], (size_t)n1 * nn * h->esz);
  }
  alloc(&h->store, (size_t)store_elems * h->esz);
  alloc((void**)&h->status, 3 * sizeof(int32_t));  // status, max |A|, max |inverted block| (bits)
  if (e != cudaSuccess) {
    bcr_destroy(h);
    return e;
  }
  *out = h;
  if (bytes) *bytes = h->factor_bytes;
  return cudaSuccess;
}

cudaError_t bcr_read_status(BcrHandle* h, int32_t* st, cudaStream_t s, double* growth) {
  uint32_t w[3] = {0, 0, 0};
  RCI_CUDA_TRY(cudaMemcpyAsync(w, h->status, sizeof(w), cudaMemcpyDeviceToHost, s));
  RCI_CUDA_TRY(cudaStreamSynchronize(s));
  *st = (int32_t)w[0];
  if (growth) {
    float a, d;
    std::memcpy(&a, &w[1], 4);
    std::memcpy(&d, &w[2], 4);
    *growth = a > 0.f ? (double)d / (double)a : 0.0;
  }
  return cudaSuccess;
}

template <typename T>
static cudaError_t factor_t(BcrHandle* h, const double2* dg, const double2* cx, const double2* cy,
                            cudaStream_t s) {
  const int nx = h->nx, ny = h->ny;
  const int64_t nn = (int64_t)ny * ny;
  const int m0 = (int)h->m[0];
  const int n1 = (nx + 1) / 2;
  RCI_CUDA_TRY(cudaMemsetAsync(h->status, 0, 3 * sizeof(int32_t), s));
  uint32_t* maxabs = reinterpret_cast<uint32_t*>(h->status) + 1;
  {
    const int64_t N = (int64_t)nx * ny;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(N, 256), 4 * 152);
    coeff_maxabs_kernel<<<grid, 256, 0, s>>>(dg, cx, cy, N, maxabs);
    rci_note_launch();
    RCI_CUDA_TRY(cudaGetLastError());
  }
  auto tdl = (cplx<T>*)h->tdl;
  auto tdinv = (cplx<T>*)h->tdinv;
  auto tdu = (cplx<T>*)h->tdu;
  auto tdu2 = (cplx<T>*)h->tdu2;
  ProfScope* l0 = new ProfScope(h->prof, PF_LEVEL0, s, 48.0 * ny * (double)ny * n1,
                                2.0 * n1 * (double)nn * sizeof(cplx<T>), 2);
  if (m0 > 0) {
    size_t tsm = TRI_WARPS * tri_smem_per_warp<T>(ny);
    if (tsm > 48 * 1024)
      RCI_CUDA_TRY(cudaFuncSetAttribute(tri_factor_kernel<T>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm));
    tri_factor_kernel<T><<<(unsigned)ceil_div(m0, TRI_WARPS), 32 * TRI_WARPS, tsm, s>>>(
        dg, cy, nx, ny, m0, tdl, tdinv, tdu, tdu2, h->tpiv, h->status);
    rci_note_launch();
    RCI_CUDA_TRY(cudaGetLastError());
  }
  {
    // D' and L' of the first reduced system; the stored inverses G0 are formed when a solve
    // with several right-hand sides first needs them
    const int thr = (int)ceil_div(ny, 32) * 32;
    const size_t smem = l0_smem<T>(ny);
    if (smem > 48 * 1024)
      RCI_CUDA_TRY(cudaFuncSetAttribute(level0_schur_kernel<T, 0>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // the next level's working arrays are free during level 0 and serve as scratch
    level0_schur_kernel<T, 0><<<n1, thr, smem, s>>>(dg, cx, cy, nx, ny, tdl, tdinv, tdu, tdu2,
                                                    h->tpiv, (cplx<T>*)h->Dw[0], (cplx<T>*)h->Lw[0],
                                                    (cplx<T>*)h->Dw[1], (cplx<T>*)h->Lw[1],
                                                    (cplx<T>*)h->G0);
    rci_note_launch();
    RCI_CUDA_TRY(cudaGetLastError());
    h->g0_valid = false;
  }
  delete l0;
  const cplx<T> one = mkc(T(1), T(0)), mone = mkc(T(-1), T(0)), zero = czero<T>();
  int cur = 0;
  auto store = (cplx<T>*)h->store;
  for (int l = 1; l < h->Lf; ++l) {
    const int n = (int)h->n[l], m = (int)h->m[l], nk = (int)h->n[l + 1];
    const int my = (n - 1) / 2;
    cplx<T>* D = (cplx<T>*)h->Dw[cur];
    cplx<T>* L = (cplx<T>*)h->Lw[cur];
    cplx<T>* Dn = (cplx<T>*)h->Dw[1 - cur];
    cplx<T>* Ln = (cplx<T>*)h->Lw[1 - cur];
    cplx<T>* Dinv = store + h->off[l];
    cplx<T>* X = Dinv + (int64_t)m * nn;
    cplx<T>* Y = X + (int64_t)m * nn;
    // D_r^{-1} for the odd rows (the working copy of D_r is destroyed)
    {
      ProfScope ps(h->prof, PF_INVERT, s, 8.0 * ny * (double)nn * m, 2.0 * m * nn * sizeof(cplx<T>), 1);
      RCI_CUDA_TRY(launch_gj<T>(D + nn, 2 * nn, Dinv, nn, ny, m, h->status, s, maxabs + 1,
                                !h->simt));
    }
    // X_k = Dinv_k L_{2k+1};  Y_k = Dinv_k L_{2k+2}^T
    // D'_k = D_{2k} - L_{2k} Y_{k-1} (k >= 1) - L_{2k+1}^T X_k (k < m)
    // L'_k = -L_{2k} X_{k-1} (k >= 1)
    // FP32 on the tensor cores: two launches, X and Y together, then each D' as one product
    // over K = 2 ny (written once) together with L'; otherwise five batched products.
    bool fused = false;
    if constexpr (sizeof(T) == 4) {
      if (nk >= 2 && my >= 1) {
        const double pb = (double)sizeof(cplx<T>) * nn;
        TcJob xy[2] = {};
        xy[0].nseg = 1;
        xy[0].seg[0] = TcSegment{Dinv, ny, nn, m, false, L + nn, ny, 2 * nn, m, false, ny, 0, 0, 0, m};
        xy[0].alpha = 1.f;
        xy[0].C = X;
        xy[0].ldc = ny;
        xy[0].sC = nn;
        xy[0].batch = m;
        xy[1] = xy[0];
        xy[1].seg[0] = TcSegment{Dinv, ny, nn, my, false, L + 2 * nn, ny, 2 * nn, my, true, ny, 0, 0, 0, my};
        xy[1].C = Y;
        xy[1].batch = my;
        TcJob sl[2] = {};
        sl[0].nseg = 2;
        sl[0].seg[0] = TcSegment{L, ny, 2 * nn, nk, false, Y, ny, nn, my, false, ny, 0, -1, 1, nk};
        sl[0].seg[1] = TcSegment{L + nn, ny, 2 * nn, m, true, X, ny, nn, m, false, ny, 0, 0, 0, m};
        sl[0].alpha = -1.f;
        sl[0].beta = 1.f;
        sl[0].C0 = D;
        sl[0].ldc0 = ny;
        sl[0].sC0 = 2 * nn;
        sl[0].C = Dn;
        sl[0].ldc = ny;
        sl[0].sC = nn;
        sl[0].batch = nk;
        sl[1].nseg = 1;
        sl[1].seg[0] = TcSegment{L + 2 * nn, ny, 2 * nn, nk - 1, false, X, ny, nn, m, false, ny, 0, 0, 0, nk - 1};
        sl[1].alpha = -1.f;
        sl[1].C = Ln + nn;
        sl[1].ldc = ny;
        sl[1].sC = nn;
        sl[1].batch = nk - 1;
        cudaError_t e;
        {
          ProfScope ps(h->prof, PF_GEMM, s, 8.0 * ny * (double)nn * (m + my), pb * 3.0 * (m + my), 1);
          e = h->simt ? cudaErrorNotSupported
                      : launch_tc_cgemm_tma_jobs(ny, ny, 2, xy, h->status, tc_wait_limit(), s);
        }
        if (e == cudaSuccess) {
          ProfScope ps(h->prof, PF_GEMM, s, 8.0 * ny * (double)nn * (2 * (nk - 1) + m),
                       pb * (2.0 * (nk - 1 + m) + 2.0 * nk + 3.0 * (nk - 1)), 1);
          RCI_CUDA_TRY(launch_tc_cgemm_tma_jobs(ny, ny, 2, sl, h->status, tc_wait_limit(), s));
          fused = true;
        } else if (e != cudaErrorNotSupported) {
          return e;
        }
      }
    }
    if (!fused) {
      RCI_CUDA_TRY(gemm<T>(ny, ny, ny, false, false, one, Dinv, ny, nn, L + nn, ny, 2 * nn, zero,
                           nullptr, 0, 0, X, ny, nn, m, s, h->prof, PF_GEMM, gemm_status(h)));
      RCI_CUDA_TRY(gemm<T>(ny, ny, ny, false, true, one, Dinv, ny, nn, L + 2 * nn, ny, 2 * nn, zero,
                           nullptr, 0, 0, Y, ny, nn, my, s, h->prof, PF_GEMM, gemm_status(h)));
      RCI_CUDA_TRY(cudaMemcpyAsync(Dn, D, nn * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, s));
      RCI_CUDA_TRY(gemm<T>(ny, ny, ny, false, false, mone, L + 2 * nn, ny, 2 * nn, Y, ny, nn, one,
                           D + 2 * nn, ny, 2 * nn, Dn + nn, ny, nn, nk - 1, s, h->prof, PF_GEMM,
                           gemm_status(h)));
      RCI_CUDA_TRY(gemm<T>(ny, ny, ny, true, false, mone, L + nn, ny, 2 * nn, X, ny, nn, one, Dn,
                           ny, nn, Dn, ny, nn, m, s, h->prof, PF_GEMM, gemm_status(h)));
      RCI_CUDA_TRY(gemm<T>(ny, ny, ny, false, false, mone, L + 2 * nn, ny, 2 * nn, X, ny, nn, zero,
                           nullptr, 0, 0, Ln + nn, ny, nn, nk - 1, s, h->prof, PF_GEMM, gemm_status(h)));
    }
    cur = 1 - cur;
  }
  // last single row
  {
    ProfScope ps(h->prof, PF_INVERT, s, 8.0 * ny * (double)nn, 2.0 * nn * sizeof(cplx<T>), 1);
    RCI_CUDA_TRY(launch_gj<T>((cplx<T>*)h->Dw[cur], 0, store + h->final_off, 0, ny, 1, h->status, s,
                              maxabs + 1, !h->simt));
  }
  return cudaSuccess;
}

cudaError_t bcr_factor(BcrHandle* h, const double2* dg, const double2* cx, const double2* cy,
                       cudaStream_t s) {
  return h->prec == RCI_FP64 ? factor_t<double>(h, dg, cx, cy, s)
                             : factor_t<float>(h, dg, cx, cy, s);
}

// workspace layout for nrhs right-hand sides (elements of cplx<T>):
//   t0 [m0 row] | B_l [n_l row] (l = 1..Lf) | t_l [m_l row] (l = 1..Lf-1) | P, Q [m_1 row] | xf [row]
static int64_t ws_elems(const BcrHandle* h, int nrhs) {
  int64_t row = (int64_t)h->ny * nrhs;
  int64_t tot = h->m[0] * row;
  for (int l = 1; l <= h->Lf; ++l) tot += h->n[l] * row;
  for (int l = 1; l < h->Lf; ++l) tot += h->m[l] * row;
  int64_t m1 = h->Lf > 1 ? h->m[1] : 0, m2 = h->Lf > 2 ? h->m[2] : 0;
  tot += 2 * m1 * row + 2 * m2 * row + row;  // P, Q of the odd levels, of the even levels, xf
  return tot;
}

cudaError_t bcr_reserve_ws(BcrHandle* h, int nrhs) {
  if (h->ws_nrhs >= nrhs) return cudaSuccess;
  free_ws(h);
  size_t bytes = (size_t)ws_elems(h, nrhs) * h->esz;
  RCI_CUDA_TRY(h->mem.alloc(&h->ws, bytes));
  h->ws_bytes = bytes;
  h->ws_nrhs = nrhs;
  return cudaSuccess;
}

template <typename T>
static cudaError_t solve_t(BcrHandle* h, const double2* cx, const cplx<T>* b, cplx<T>* x, int nrhs,
                           cudaStream_t s) {
  const int nx = h->nx, ny = h->ny;
  const int64_t nn = (int64_t)ny * ny;
  const int64_t row = (int64_t)ny * nrhs;
  const int m0 = (int)h->m[0], n1 = (nx + 1) / 2;
  RCI_CUDA_TRY(bcr_reserve_ws(h, nrhs));
  // carve the workspace
  cplx<T>* p = (cplx<T>*)h->ws;
  cplx<T>* t0 = p;
  p += h->m[0] * row;
  std::vector<cplx<T>*> B(h->Lf + 1, nullptr), tl(h->Lf + 1, nullptr);
  for (int l = 1; l <= h->Lf; ++l) {
    B[l] = p;
    p += h->n[l] * row;
  }
  for (int l = 1; l < h->Lf; ++l) {
    tl[l] = p;
    p += h->m[l] * row;
  }
  int64_t m1 = h->Lf > 1 ? h->m[1] : 0, m2 = h->Lf > 2 ? h->m[2] : 0;
  cplx<T>* P = p;
  p += m1 * row;
  cplx<T>* Q = p;
  p += m1 * row;
  // a second pair for the even levels: one right-hand side forms a level's rows from the P
  // and Q of the level before while it writes its own
  cplx<T>* P2 = p;
  p += m2 * row;
  cplx<T>* Q2 = p;
  p += m2 * row;
  cplx<T>* xf = p;

  auto store = (const cplx<T>*)h->store;
  const cplx<T>* G0 = (const cplx<T>*)h->G0;
  const cplx<T> one = mkc(T(1), T(0)), mone = mkc(T(-1), T(0)), zero = czero<T>();

  // level 0: the tridiagonal factors twice for one right-hand side (dense inverses G0 for
  // several); levels >= 1: Dinv, X, Y forward and X, Y backward
  double sbytes = nrhs == 1 ? 2.0 * m0 * 5.0 * ny * sizeof(cplx<T>) : 2.0 * m0 * (double)nn * sizeof(cplx<T>);
  double sflops = nrhs == 1 ? 2.0 * 30.0 * m0 * (double)ny : 2.0 * 8.0 * m0 * (double)nn * nrhs;
  for (int l = 1; l < h->Lf; ++l) {
    sbytes += 5.0 * h->m[l] * (double)nn * sizeof(cplx<T>);
    sflops += 5.0 * 8.0 * h->m[l] * (double)nn * nrhs;
  }
  sbytes += (double)nn * sizeof(cplx<T>) + 2.0 * nx * (double)ny * nrhs * sizeof(cplx<T>);
  ProfScope ps(h->prof, PF_SOLVE, s, sflops, sbytes, 0);
  // kernels this solve launches (level-0 pair, per dense level forward and backward, the
  // single remaining row); several right-hand sides run the level products as GEMMs
  {
    const int dense = h->Lf - 1, l0 = m0 > 0 ? 1 : 0;
    ps.nl = nrhs == 1 ? l0 + 1 + dense + 1 + dense + 1
                      : l0 + 1 + 4 * dense + 1 + 3 * dense + 1 + l0;
  }

  if (nrhs == 1) {
    if (ny % vec16<T>::per != 0 || ny > 256 * vec16<T>::per)
      return cudaErrorInvalidValue;  // (grid creation keeps ny within these limits)
    const int smax = (int)ceil_div(ny, 32 * vec16<T>::per);
    const unsigned nch = (unsigned)ceil_div(ny, RC);
    const size_t red_smem = (size_t)2 * CH_WARPS * RC * sizeof(cplx<T>);
#define RCI_SMAX_DISPATCH(KERNEL, GRID, SMEM, ...)                                   \
  do {                                                                               \
    switch (smax) {                                                                  \
      case 1: KERNEL<T, 1><<<GRID, CH_THREADS, SMEM, s>>>(__VA_ARGS__); break;       \
      case 2: KERNEL<T, 2><<<GRID, CH_THREADS, SMEM, s>>>(__VA_ARGS__); break;       \
      case 3: KERNEL<T, 3><<<GRID, CH_THREADS, SMEM, s>>>(__VA_ARGS__); break;       \
      case 4: KERNEL<T, 4><<<GRID, CH_THREADS, SMEM, s>>>(__VA_ARGS__); break;       \
      case 5: KERNEL<T, 5><<<GRID, CH_THREADS, SMEM, s>>>(__VA_ARGS__); break;       \
      case 6: KERNEL<T, 6><<<GRID, CH_THREADS, SMEM, s>>>(__VA_ARGS__); break;       \
      case 7: KERNEL<T, 7><<<GRID, CH_THREADS, SMEM, s>>>(__VA_ARGS__); break;       \
      default: KERNEL<T, 8><<<GRID, CH_THREADS, SMEM, s>>>(__VA_ARGS__); break;      \
    }                                                                                \
    rci_note_launch();                                                               \
    RCI_CUDA_TRY(cudaGetLastError());                                                \
  } while (0)
    // the chunked level-0 backward pass reads b while other blocks write x: no aliasing
    const cplx<T>* bsrc = b;
    if ((const void*)b == (const void*)x) return cudaErrorInvalidValue;
    // ---- level 0 forward: t0[k] = T_{2k+1}^{-1} b[2k+1] by tridiagonal sweeps
    const size_t trs_smem = TRS_WARPS * trs_smem_per_warp<T>(ny);
    auto trs_attr = [&](auto kern) -> cudaError_t {
      return trs_smem > 48 * 1024 ? cudaFuncSetAttribute(kern,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)trs_smem)
                                  : cudaSuccess;
    };
    if (m0 > 0) {
      RCI_CUDA_TRY(trs_attr(tri_rows_solve_kernel<T, false>));
      tri_rows_solve_kernel<T, false><<<(unsigned)ceil_div(m0, TRS_WARPS), 32 * TRS_WARPS,
                                        trs_smem, s>>>(
          (const cplx<T>*)h->tdl, (const cplx<T>*)h->tdinv, (const cplx<T>*)h->tdu,
          (const cplx<T>*)h->tdu2, h->tpiv, bsrc, nullptr, cx, t0, nx, ny, m0);
      rci_note_launch();
      RCI_CUDA_TRY(cudaGetLastError());
    }
    {
      int64_t nt = (int64_t)n1 * row;
      keep0_kernel<T><<<(unsigned)ceil_div(nt, 256), 256, 0, s>>>(bsrc, t0, cx, B[1], nx, ny, n1, 1);
      rci_note_launch();
      RCI_CUDA_TRY(cudaGetLastError());
    }
    // ---- dense levels forward: level 1 from the kept rows of level 0; every later level forms
    // its rows from the level before (the kept-row update fused into its forward kernel), the
    // P and Q of odd levels in (P, Q), of even levels in (P2, Q2)
    auto Pl = [&](int l) { return (l & 1) ? P : P2; };
    auto Ql = [&](int l) { return (l & 1) ? Q : Q2; };
    for (int l = 1; l < h->Lf; ++l) {
      const int n = (int)h->n[l], m = (int)h->m[l];
      const cplx<T>* Dinv = store + h->off[l];
      const cplx<T>* X = Dinv + (int64_t)m * nn;
      const cplx<T>* Y = X + (int64_t)m * nn;
      if (l == 1) {
        RCI_SMAX_DISPATCH(fwd_chunk_kernel, dim3(m, nch), ny * sizeof(cplx<T>) + red_smem, Dinv,
                          X, Y, B[1], tl[1], Pl(1), Ql(1), n, ny);
      } else {
        RCI_SMAX_DISPATCH(fwd_keep_chunk_kernel, dim3((unsigned)h->n[l + 1], nch),
                          ny * sizeof(cplx<T>) + red_smem, Dinv, X, Y, B[l - 1], Pl(l - 1),
                          Ql(l - 1), (int)h->m[l - 1], B[l], tl[l], Pl(l), Ql(l), n, ny);
      }
    }
    // ---- single remaining row (from the level before it when there is one, written straight
    // to B[Lf], which nothing reads as input then)
    if (h->Lf >= 2) {
      const int lp = h->Lf - 1;
      RCI_SMAX_DISPATCH(mv_keep_chunk_kernel, dim3(1, nch), ny * sizeof(cplx<T>),
                        store + h->final_off, B[lp], Pl(lp), Ql(lp), (int)h->m[lp], B[h->Lf], ny);
    } else {
      RCI_SMAX_DISPATCH(mv_chunk_kernel, dim3(1, nch), ny * sizeof(cplx<T>), store + h->final_off,
                        B[h->Lf], (int64_t)0, (int64_t)0, xf, ny);
      RCI_CUDA_TRY(cudaMemcpyAsync(B[h->Lf], xf, row * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, s));
    }
    // ---- dense levels backward (the solution of level l overwrites B[l])
    for (int l = h->Lf - 1; l >= 1; --l) {
      const int n = (int)h->n[l], m = (int)h->m[l], nk = (int)h->n[l + 1];
      const cplx<T>* Dinv = store + h->off[l];
      const cplx<T>* X = Dinv + (int64_t)m * nn;
      const cplx<T>* Y = X + (int64_t)m * nn;
      RCI_SMAX_DISPATCH(bwd_chunk_kernel, dim3(nk, nch), 3 * ny * sizeof(cplx<T>), X, Y, tl[l],
                        B[l + 1], B[l], n, m, ny);
    }
    // ---- level 0 backward by tridiagonal sweeps (and the kept rows copied)
    RCI_CUDA_TRY(trs_attr(tri_rows_solve_kernel<T, true>));
    tri_rows_solve_kernel<T, true><<<(unsigned)ceil_div(n1, TRS_WARPS), 32 * TRS_WARPS,
                                     trs_smem, s>>>(
        (const cplx<T>*)h->tdl, (const cplx<T>*)h->tdinv, (const cplx<T>*)h->tdu,
        (const cplx<T>*)h->tdu2, h->tpiv, bsrc, B[1], cx, x, nx, ny, n1);
    rci_note_launch();
    RCI_CUDA_TRY(cudaGetLastError());
#undef RCI_SMAX_DISPATCH
    return cudaSuccess;
  }

  // ================= several right-hand sides: batched GEMMs per level
  // ---- the stored inverses of level 0, formed once per factorisation
  if (m0 > 0 && !h->g0_valid) {
    const int thr = (int)ceil_div(ny, 32) * 32;
    const size_t smem = l0_smem<T>(ny);
    if (smem > 48 * 1024)
      RCI_CUDA_TRY(cudaFuncSetAttribute(level0_schur_kernel<T, 1>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cplx<T>* g0w = (cplx<T>*)h->G0;
    level0_schur_kernel<T, 1><<<m0, thr, smem, s>>>(nullptr, nullptr, nullptr, nx, ny,
                                                    (const cplx<T>*)h->tdl, (const cplx<T>*)h->tdinv,
                                                    (const cplx<T>*)h->tdu, (const cplx<T>*)h->tdu2,
                                                    h->tpiv, g0w, g0w, g0w, g0w, g0w);
    rci_note_launch();
    RCI_CUDA_TRY(cudaGetLastError());
    h->g0_valid = true;
  }
  // ---- level 0 forward: t0[k] = T_{2k+1}^{-1} b[2k+1] with the stored inverses
  if (m0 > 0)
    RCI_CUDA_TRY(gemm<T>(ny, nrhs, ny, false, false, one, G0, ny, nn, b + row, nrhs, 2 * row, zero,
                         nullptr, 0, 0, t0, nrhs, row, m0, s, nullptr, PF_SOLVE, gemm_status(h)));
  {
    int64_t nt = (int64_t)n1 * row;
    keep0_kernel<T><<<(unsigned)ceil_div(nt, 256), 256, 0, s>>>(b, t0, cx, B[1], nx, ny, n1, nrhs);
    rci_note_launch();
    RCI_CUDA_TRY(cudaGetLastError());
  }
  // ---- dense levels forward
  for (int l = 1; l < h->Lf; ++l) {
    const int n = (int)h->n[l], m = (int)h->m[l], nk = (int)h->n[l + 1];
    const int my = (n - 1) / 2;
    const cplx<T>* Dinv = store + h->off[l];
    const cplx<T>* X = Dinv + (int64_t)m * nn;
    const cplx<T>* Y = X + (int64_t)m * nn;
    const cplx<T>* Bodd = B[l] + row;
    RCI_CUDA_TRY(gemm<T>(ny, nrhs, ny, false, false, one, Dinv, ny, nn, Bodd, nrhs, 2 * row, zero,
                         nullptr, 0, 0, tl[l], nrhs, row, m, s, nullptr, PF_SOLVE, gemm_status(h)));
    RCI_CUDA_TRY(gemm<T>(ny, nrhs, ny, true, false, one, X, ny, nn, Bodd, nrhs, 2 * row, zero,
                         nullptr, 0, 0, P, nrhs, row, m, s, nullptr, PF_SOLVE, gemm_status(h)));
    RCI_CUDA_TRY(gemm<T>(ny, nrhs, ny, true, false, one, Y, ny, nn, Bodd, nrhs, 2 * row, zero,
                         nullptr, 0, 0, Q, nrhs, row, my, s, nullptr, PF_SOLVE, gemm_status(h)));
    int64_t nt = (int64_t)nk * row;
    keep_kernel<T><<<(unsigned)ceil_div(nt, 256), 256, 0, s>>>(B[l], P, Q, B[l + 1], m, nk, row);
    rci_note_launch();
    RCI_CUDA_TRY(cudaGetLastError());
  }
  // ---- single remaining row
  RCI_CUDA_TRY(gemm<T>(ny, nrhs, ny, false, false, one, store + h->final_off, ny, 0, B[h->Lf], nrhs,
                       0, zero, nullptr, 0, 0, xf, nrhs, 0, 1, s, nullptr, PF_SOLVE, gemm_status(h)));
  RCI_CUDA_TRY(cudaMemcpyAsync(B[h->Lf], xf, row * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, s));
  // ---- dense levels backward (the solution of level l overwrites B[l])
  for (int l = h->Lf - 1; l >= 1; --l) {
    const int n = (int)h->n[l], m = (int)h->m[l], nk = (int)h->n[l + 1];
    const int my = (n - 1) / 2;
    const cplx<T>* Dinv = store + h->off[l];
    const cplx<T>* X = Dinv + (int64_t)m * nn;
    const cplx<T>* Y = X + (int64_t)m * nn;
    int64_t nt = (int64_t)nk * row;
    copy_kept_kernel<T><<<(unsigned)ceil_div(nt, 256), 256, 0, s>>>(B[l + 1], B[l], nk, row);
    rci_note_launch();
    RCI_CUDA_TRY(cudaGetLastError());
    RCI_CUDA_TRY(gemm<T>(ny, nrhs, ny, false, false, mone, X, ny, nn, B[l + 1], nrhs, row, one,
                         tl[l], nrhs, row, B[l] + row, nrhs, 2 * row, m, s, nullptr, PF_SOLVE, gemm_status(h)));
    RCI_CUDA_TRY(gemm<T>(ny, nrhs, ny, false, false, mone, Y, ny, nn, B[l + 1] + row, nrhs, row,
                         one, B[l] + row, nrhs, 2 * row, B[l] + row, nrhs, 2 * row, my, s, nullptr, PF_SOLVE, gemm_status(h)));
  }
  // ---- level 0 backward: x[2k+1] = T^{-1}(b[2k+1] - couplings x), stored inverses
  {
    int64_t nt = (int64_t)n1 * row;
    // t0 (no longer needed) holds the eliminated rows' right-hand sides
    bwd0_rhs_kernel<T><<<(unsigned)ceil_div(nt, 256), 256, 0, s>>>(b, B[1], cx, x, t0, nx, ny, n1,
                                                                    nrhs);
    rci_note_launch();
    RCI_CUDA_TRY(cudaGetLastError());
    if (m0 > 0)
      RCI_CUDA_TRY(gemm<T>(ny, nrhs, ny, false, false, one, G0, ny, nn, t0, nrhs, row, zero,
                           nullptr, 0, 0, x + row, nrhs, 2 * row, m0, s, nullptr, PF_SOLVE, gemm_status(h)));
  }
  return cudaSuccess;
}

cudaError_t bcr_solve(BcrHandle* h, const double2* cx, const void* b, void* x, int nrhs,
                      cudaStream_t s) {
  if (nrhs < 1) return cudaErrorInvalidValue;
  if (h->prec == RCI_FP64)
    return solve_t<double>(h, cx, (const double2*)b, (double2*)x, nrhs, s);
  return solve_t<float>(h, cx, (const float2*)b, (float2*)x, nrhs, s);
}

cudaError_t bcr_block_inverse(const void* src, void* out, int n, int batch, int prec, int kernel,
                              int32_t* status, cudaStream_t s) {
  const int64_t nn = (int64_t)n * n;
  if (prec == RCI_FP64) {
    if (kernel == 2) return cudaErrorInvalidValue;
    return launch_gj<double>((double2*)src, nn, (double2*)out, nn, n, batch, status, s);
  }
  if (kernel == 1) return launch_gj_simt<float>((float2*)src, nn, (float2*)out, nn, n, batch, status, s);
  if (kernel == 2) return launch_tc_gj((const float2*)src, nn, (float2*)out, nn, n, batch, status, s);
  return launch_gj<float>((float2*)src, nn, (float2*)out, nn, n, batch, status, s);
}

cudaError_t bcr_gemm(int M, int N, int K, bool ta, bool tb, double alpha, const void* A,
                     int64_t lda, int64_t sA, const void* B, int64_t ldb, int64_t sB, double beta,
                     const void* C0, int64_t ldc0, int64_t sC0, void* C, int64_t ldc, int64_t sC,
                     int batch, int prec, int kernel, int32_t* status, cudaStream_t s) {
  if (prec == RCI_FP64) {
    if (kernel == 1 || kernel == 2) return cudaErrorInvalidValue;
    const cplx<double> al{alpha, 0.0}, be{beta, 0.0};
    return gemm<double>(M, N, K, ta, tb, al, (const double2*)A, lda, sA, (const double2*)B, ldb,
                        sB, be, (const double2*)C0, ldc0, sC0, (double2*)C, ldc, sC, batch, s);
  }
  const float2 al = make_float2((float)alpha, 0.f), be = make_float2((float)beta, 0.f);
  const float2 *a = (const float2*)A, *b = (const float2*)B, *c0 = (const float2*)C0;
  float2* c = (float2*)C;
  switch (kernel) {
    case 1:
      return launch_tc_cgemm(M, N, K, ta, tb, al, a, lda, sA, b, ldb, sB, be, c0, ldc0, sC0, c, ldc,
                             sC, batch, status, s, 1);
    case 2: {
      const cudaError_t e = launch_tc_cgemm_tma(M, N, K, ta, tb, (float)alpha, a, lda, sA, b, ldb, sB,
                                                (float)beta, c0, ldc0, sC0, c, ldc, sC, batch,
                                                status, tc_wait_limit(), s);
      return e == cudaErrorNotSupported ? cudaErrorInvalidValue : e;
    }
    case 3:  // SIMT: no status word, so the dispatch keeps off the tensor cores
      return gemm<float>(M, N, K, ta, tb, al, a, lda, sA, b, ldb, sB, be, c0, ldc0, sC0, c, ldc, sC,
                         batch, s);
    default:
      return gemm<float>(M, N, K, ta, tb, al, a, lda, sA, b, ldb, sB, be, c0, ldc0, sC0, c, ldc, sC,
                         batch, s, nullptr, PF_GEMM, status);
  }
}
