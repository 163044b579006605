// Linear-algebra kernels of the Newton step: block-CSR SpMV with symmetric Dirichlet
// elimination, Jacobi / 3x3 block-Jacobi preconditioned conjugate gradients, the free-dof
// residual norm and the displacement update (paper Eq. Stiffness_mat; the paper's
// identity-row elimination of App. E is made symmetric here: rows and columns of fixed dofs
// are dropped, the diagonal set to one).
//
// Reductions are deterministic: every CTA writes a partial sum, and the last CTA to finish
// (ticket counter, no waiting) adds the partials in index order and derives the scalars
// (alpha, beta) that the next kernel reads from device memory, so a CG iteration needs no
// host round trip and can be captured in a CUDA graph.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "solver.h"

namespace hfe {
namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename R>
__device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block reduction of up to two doubles; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  if (w == 0) {
    a = (l < nw) ? sa[l] : 0.0;
    b = (l < nw) ? sb[l] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

// Last-CTA reduction of the partials; returns true in every thread of the last CTA, which
// then holds the totals in t0 / t1 (thread 0 only).
__device__ __forceinline__ bool last_block_reduce(double pa, double pb, double* part, unsigned* ticket,
                                                  double& t0, double& t1) {
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = pa;
    part[2 * blockIdx.x + 1] = pb;
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double a = 0.0, b = 0.0;
  // fixed-order reduction: thread k sums partials k, k + blockDim, ... then a block reduction
  for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
    a += __ldcg(part + 2 * k);
    b += __ldcg(part + 2 * k + 1);
  }
  block_sum2(a, b);
  t0 = a;
  t1 = b;
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// y = Kt x with Kt the matrix whose fixed rows/columns are dropped and whose fixed diagonal is 1.
// A warp serves two block rows per pass, one lane per 3x3 block of each (rows with more than
// 32 blocks loop): the lane loads the block's column, the three x entries it multiplies and
// its 9 values (the warp's value loads cover the row's contiguous 36-byte blocks), then the
// warp reduces the six partial row sums.  This standalone form serves the exported SpMV, the
// tangent predictor and the chunked CG (pcg_persistent = 0); the one-launch CG solve runs its
// own eight-lanes-per-row SpMV.  COLMASK = false skips the column mask: inside CG the fixed
// components of p are exactly zero (r, z and p start at zero there and stay zero).
// Optionally accumulates x.y (FP64) into a last-CTA reduction that sets alpha = rz / (p.Ap).
template <typename R, bool COLMASK>
__global__ void __launch_bounds__(kBlock) spmv_kernel(const int64_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ cols,
                                                      const R* __restrict__ vals,
                                                      const uint8_t* __restrict__ freem,
                                                      const R* __restrict__ x, R* __restrict__ y,
                                                      int64_t n_nodes, PcgScalars* sc, double* part) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (kBlock / 32);
  const int64_t w = (int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
  double dot = 0.0;
  // each warp takes two rows per pass (rows w + 2k nwarps and w + (2k+1) nwarps): two
  // independent load chains in flight per lane
  for (int64_t r0 = w; r0 < n_nodes; r0 += 2 * nwarps) {
    const int64_t r1 = r0 + nwarps;
    const bool has1 = r1 < n_nodes;
    const int64_t b0 = rowptr[r0], e0 = rowptr[r0 + 1];
    const int64_t b1 = has1 ? rowptr[r1] : 0, e1 = has1 ? rowptr[r1 + 1] : 0;
    const int nb0 = (int)(e0 - b0), nb1 = (int)(e1 - b1);
    R a[2][3] = {{R(0), R(0), R(0)}, {R(0), R(0), R(0)}};
    const int nmax = nb0 > nb1 ? nb0 : nb1;
    for (int j = lane; j < nmax; j += 32) {
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int nb = t == 0 ? nb0 : nb1;
        if (j < nb) {
          const int64_t blk = (t == 0 ? b0 : b1) + j;
          const int64_t col = cols[blk];
          const R* v = vals + blk * 9;
          R x0 = x[3 * col], x1 = x[3 * col + 1], x2 = x[3 * col + 2];
          if (COLMASK) {
            x0 = freem[3 * col] ? x0 : R(0);
            x1 = freem[3 * col + 1] ? x1 : R(0);
            x2 = freem[3 * col + 2] ? x2 : R(0);
          }
          a[t][0] += v[0] * x0 + v[1] * x1 + v[2] * x2;
          a[t][1] += v[3] * x0 + v[4] * x1 + v[5] * x2;
          a[t][2] += v[6] * x0 + v[7] * x1 + v[8] * x2;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int i = 0; i < 3; ++i) a[t][i] = warp_sum_r(a[t][i]);
    if (lane < 6) {
      const int t = lane / 3, i = lane % 3;
      if (t == 0 || has1) {
        const int64_t d = 3 * (t == 0 ? r0 : r1) + i;
        const R o = t == 0 ? (i == 0 ? a[0][0] : (i == 1 ? a[0][1] : a[0][2]))
                           : (i == 0 ? a[1][0] : (i == 1 ? a[1][1] : a[1][2]));
        const R xd = x[d];
        const R out = freem[d] ? o : (COLMASK ? xd : R(0));
        y[d] = out;
        dot += (double)xd * (double)out;
      }
    }
  }
  if (sc == nullptr) return;
  double dummy = 0.0;
  block_sum2(dot, dummy);
  double tot, t1;
  if (last_block_reduce(dot, 0.0, part, &sc->ticket, tot, t1) && threadIdx.x == 0) {
    sc->pq = tot;
    const bool ok = (tot > 0.0) && isfinite(tot) && isfinite(sc->rz);
    sc->alpha = (ok && !sc->done) ? sc->rz / tot : 0.0;
    if (!ok && !sc->done && sc->rz > 0.0) sc->breakdown = 1;
  }
}

// x += alpha p; r -= alpha q; z = M^-1 r; partial (r.z, r.r); last CTA: beta = rz_new / rz.
template <typename R>
__global__ void __launch_bounds__(kBlock) pcg_update_kernel(R* __restrict__ x, R* __restrict__ r, R* __restrict__ z,
                                                            const R* __restrict__ p, const R* __restrict__ q,
                                                            const R* __restrict__ minv, int block3,
                                                            int64_t n_nodes, PcgScalars* sc, double* part) {
  double rz = 0.0, rr = 0.0;
  const R al = (R)sc->alpha;
  for (int64_t n = (int64_t)blockIdx.x * kBlock + threadIdx.x; n < n_nodes; n += (int64_t)gridDim.x * kBlock) {
    R rv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int64_t d = 3 * n + i;
      x[d] += al * p[d];
      rv[i] = r[d] - al * q[d];
      r[d] = rv[i];
    }
    R zv[3];
    if (block3) {
      const R* M = minv + 9 * n;
#pragma unroll
      for (int i = 0; i < 3; ++i) zv[i] = M[3 * i] * rv[0] + M[3 * i + 1] * rv[1] + M[3 * i + 2] * rv[2];
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) zv[i] = minv[3 * n + i] * rv[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      z[3 * n + i] = zv[i];
      rz += (double)rv[i] * (double)zv[i];
      rr += (double)rv[i] * (double)rv[i];
    }
  }
  block_sum2(rz, rr);
  double trz, trr;
  if (last_block_reduce(rz, rr, part, &sc->ticket, trz, trr) && threadIdx.x == 0) {
    if (!sc->done) {
      const double old = sc->rz;
      sc->beta = (old > 0.0) ? trz / old : 0.0;
      sc->rz = trz;
      sc->rr = trr;
      sc->iters += 1;
      if (!isfinite(trz) || !isfinite(trr)) sc->breakdown = 1;
      if (trr <= sc->target) sc->done = 1;
    }
  }
}

// p = z + beta p
template <typename R>
__global__ void __launch_bounds__(kBlock) pcg_p_kernel(R* __restrict__ p, const R* __restrict__ z, int64_t n_dof,
                                                       const PcgScalars* sc) {
  const int64_t d = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (d < n_dof) p[d] = z[d] + (R)sc->beta * p[d];
}

// r = b (fixed components zeroed), x = 0, z = M^-1 r, p = z; rz = r.z, rr = r.r.
template <typename R>
__global__ void __launch_bounds__(kBlock) pcg_init_kernel(const double* __restrict__ b, const uint8_t* __restrict__ freem,
                                                          double bscale, R* __restrict__ x, R* __restrict__ r,
                                                          R* __restrict__ z, R* __restrict__ p,
                                                          const R* __restrict__ minv, int block3, int64_t n_nodes,
                                                          PcgScalars* sc, double* part) {
  double rz = 0.0, rr = 0.0;
  for (int64_t n = (int64_t)blockIdx.x * kBlock + threadIdx.x; n < n_nodes; n += (int64_t)gridDim.x * kBlock) {
    R rv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int64_t d = 3 * n + i;
      rv[i] = freem[d] ? (R)(bscale * b[d]) : R(0);
      r[d] = rv[i];
      x[d] = R(0);
    }
    R zv[3];
    if (block3) {
      const R* M = minv + 9 * n;
#pragma unroll
      for (int i = 0; i < 3; ++i) zv[i] = M[3 * i] * rv[0] + M[3 * i + 1] * rv[1] + M[3 * i + 2] * rv[2];
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) zv[i] = minv[3 * n + i] * rv[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      z[3 * n + i] = zv[i];
      p[3 * n + i] = zv[i];
      rz += (double)rv[i] * (double)zv[i];
      rr += (double)rv[i] * (double)rv[i];
    }
  }
  block_sum2(rz, rr);
  double trz, trr;
  if (last_block_reduce(rz, rr, part, &sc->ticket, trz, trr) && threadIdx.x == 0) {
    sc->rz = trz;
    sc->rr = trr;
    sc->rr0 = trr;
    sc->alpha = 0.0;
    sc->beta = 0.0;
    sc->iters = 0;
    sc->breakdown = (isfinite(trz) && isfinite(trr)) ? 0 : 1;
    sc->target = sc->target * trr;     // the host stores rtol^2 here before the init kernel
    sc->done = (trr <= sc->target) ? 1 : 0;
  }
}

// Preconditioner from the diagonal blocks of Kt (fixed rows/columns dropped, unit diagonal):
// Jacobi = 1 / diag, block3 = inverse of the 3x3 diagonal block (cofactors, FP64).
__device__ __forceinline__ double surrogate_inv(double d) {
  const double a = fabs(d);
  return (a > 0.0 && isfinite(a)) ? 1.0 / a : 1.0;
}

template <typename R>
__global__ void precond_kernel(const R* __restrict__ vals, const int64_t* __restrict__ diag_slot,
                               const uint8_t* __restrict__ freem, R* __restrict__ minv, int block3,
                               int64_t n_nodes, int* bad) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  const R* B = vals + 9 * diag_slot[n];
  double M[3][3];
  bool f[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) f[i] = freem[3 * n + i] != 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i][j] = (f[i] && f[j]) ? (double)B[3 * i + j] : (i == j ? 1.0 : 0.0);
  // A block (or diagonal entry) that is not positive definite is counted in *bad and replaced by
  // the positive surrogate diag(1/|M_ii|), so that the preconditioner stays SPD; the host either
  // rejects the solve or, for a Newton correction that may stop at negative curvature, goes on.
  if (!block3) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (!(M[i][i] > 0.0)) atomicAdd(bad, 1);
      minv[3 * n + i] = (R)surrogate_inv(M[i][i]);
    }
    return;
  }
  double c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1];
  double c01 = M[1][2] * M[2][0] - M[1][0] * M[2][2];
  double c02 = M[1][0] * M[2][1] - M[1][1] * M[2][0];
  double det = M[0][0] * c00 + M[0][1] * c01 + M[0][2] * c02;
  // Sylvester's criterion on the leading minors
  if (!(M[0][0] > 0.0) || !(M[0][0] * M[1][1] - M[0][1] * M[1][0] > 0.0) || !(det > 0.0)) {
    atomicAdd(bad, 1);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) minv[9 * n + 3 * i + j] = (R)(i == j ? surrogate_inv(M[i][i]) : 0.0);
    return;
  }
  double id = 1.0 / det;
  double I[3][3];
  I[0][0] = c00 * id;
  I[1][0] = c01 * id;
  I[2][0] = c02 * id;
  I[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) * id;
  I[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) * id;
  I[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) * id;
  I[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) * id;
  I[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) * id;
  I[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) * id;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) minv[9 * n + 3 * i + j] = (R)I[i][j];
}

// ||R_free||^2 (FP64, deterministic) into sc->rr via the last-CTA reduction.
__global__ void __launch_bounds__(kBlock) free_norm_kernel(const double* __restrict__ R_, const uint8_t* __restrict__ freem,
                                                           int64_t n_dof, PcgScalars* sc, double* part, double* out) {
  const int64_t d0 = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  double s = 0.0, nf = 0.0;
  for (int64_t d = d0; d < n_dof; d += (int64_t)gridDim.x * kBlock) {
    double v = freem[d] ? R_[d] : 0.0;
    s += v * v;
    if (!isfinite(v)) nf += 1.0;
  }
  block_sum2(s, nf);
  double ts, tn;
  if (last_block_reduce(s, nf, part, &sc->ticket, ts, tn) && threadIdx.x == 0) {
    sc->norm2 = ts;
    sc->nonfinite = tn;
    if (out != nullptr) *out = sqrt(ts);
  }
}

template <typename R>
__global__ void add_update_kernel(double* __restrict__ u, const R* __restrict__ x, const uint8_t* __restrict__ freem,
                                  double c, int64_t n_dof) {
  const int64_t d = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (d < n_dof && freem[d]) u[d] += c * (double)x[d];
}

__global__ void set_dirichlet_kernel(double* __restrict__ u, const int64_t* __restrict__ dof,
                                     const double* __restrict__ val, double t, int64_t n_fixed) {
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i < n_fixed) u[dof[i]] = t * val[i];
}

template <typename A, typename B>
__global__ void convert_kernel(const A* __restrict__ a, B* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i < n) b[i] = (B)a[i];
}

// b = -(R + K du_D - dt f_ext) on free dofs, 0 on fixed dofs (tangent predictor right-hand side)
template <typename R>
__global__ void predictor_rhs_kernel(const double* __restrict__ R_, const R* __restrict__ Kd, const double* __restrict__ f_ext,
                                     double dt, const uint8_t* __restrict__ freem, double* __restrict__ b, int64_t n_dof) {
  const int64_t d = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (d >= n_dof) return;
  double v = R_[d] + (double)Kd[d] - (f_ext ? dt * f_ext[d] : 0.0);
  b[d] = freem[d] ? -v : 0.0;
}


// ---------------------------------------------------------------------------------------
// Persistent PCG: the whole solve in one cooperative launch.  The rows (nodes) are split in
// contiguous ranges over the CTAs; every global quantity (p.q, r.z, r.r) is a fixed-order
// sum of per-CTA partials that every CTA recomputes after a grid barrier, so all CTAs take
// the same decisions and the result is deterministic.  Two barriers per iteration: the
// search direction p = z + beta p_prev is formed on the fly inside the SpMV (for the
// gathered columns from z and the previous direction, for the own rows also stored), with
// p_prev and p in two buffers that swap each iteration.
// Grid barrier fused with a reduction: every CTA publishes its partial pair in part, the
// last CTA to arrive sums all pairs in CTA order (the same fixed order whichever CTA is
// last) into gs.tot and releases the others, who read the totals.  Waits are bounded by
// spin_limit polls; returns false once any wait has run out (sticky), after which every CTA
// leaves the solve (a CTA released just before another gave up meets the next barrier,
// whose count can no longer complete, and gives up there).
__device__ __forceinline__ bool grid_allreduce(GridSync* gs, const double* part, double& t0, double& t1,
                                               unsigned long long spin_limit) {
  __shared__ int s_last, s_ok;
  __shared__ double s_t0, s_t1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g0 = *(volatile unsigned*)&gs->gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&gs->count, 1u);
    s_last = arrived == gridDim.x - 1;
    if (!s_last) {
      unsigned long long spins = 0;
      unsigned ns = 32;
      while (*(volatile unsigned*)&gs->gen == g0) {
        if (++spins > spin_limit) {
          atomicExch(&gs->timeout, 1);
          break;
        }
        __nanosleep(ns);
        if (ns < 256) ns *= 2;
      }
      __threadfence();
    }
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double a = 0.0, b = 0.0;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += kBlock) {
      a += __ldcg(part + 2 * k);
      b += __ldcg(part + 2 * k + 1);
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) {
      gs->tot[0] = a;
      gs->tot[1] = b;
      gs->count = 0u;
      __threadfence();
      atomicAdd(&gs->gen, 1u);
    }
  }
  if (threadIdx.x == 0) {
    s_t0 = __ldcg(&gs->tot[0]);
    s_t1 = __ldcg(&gs->tot[1]);
    s_ok = *(volatile int*)&gs->timeout == 0;
  }
  __syncthreads();
  t0 = s_t0;
  t1 = s_t1;
  return s_ok != 0;
}

// out = K in on the rows [n0, n1) (fixed rows 0; in is zero on fixed dofs), returning this
// thread's share of out . w over those rows.  Eight lanes per block row (four rows per warp
// and pass): each lane takes two blocks of a 16-block chunk of its row and issues the
// column, value and x loads of both before the arithmetic; the row sum is a three-level
// shuffle within the eight lanes.  (A warp per row, one block per lane and a five-level
// shuffle per row left the memory pipeline short of loads in flight: 0.38 against 0.34 ms
// per CG iteration at 3.09M dofs.)
template <typename R>
__device__ __forceinline__ double spmv_range(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ cols,
                                             const R* __restrict__ vals, const uint8_t* __restrict__ freem,
                                             const R* in, R* out, const R* w, int64_t n0, int64_t n1) {
  constexpr int kG = 8;                  // lanes per block row
  constexpr int kRows = 32 / kG;         // block rows per warp and pass
  constexpr int kWarps = kBlock / 32;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int grp = lane / kG, gl = lane % kG;
  double dot = 0.0;
  for (int64_t base = n0 + (int64_t)warp * kRows; base < n1; base += (int64_t)kWarps * kRows) {
    const int64_t r = base + grp;
    const bool has = r < n1;
    int64_t b = 0, e = 0;
    if (has) {
      b = rowptr[r];
      e = rowptr[r + 1];
    }
    R a0 = R(0), a1 = R(0), a2 = R(0);
    for (int64_t c = b; c < e; c += 2 * kG) {
      // up to four blocks per lane, all loads issued before the arithmetic
      int64_t col[2];
      bool ok[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int64_t k = c + gl + t * kG;
        ok[t] = k < e;
        col[t] = ok[t] ? (int64_t)cols[k] : 0;
      }
      R v[2][9], x[2][3];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int64_t k = c + gl + t * kG;
#pragma unroll
        for (int q = 0; q < 9; ++q) v[t][q] = ok[t] ? vals[k * 9 + q] : R(0);
#pragma unroll
        for (int q = 0; q < 3; ++q) x[t][q] = ok[t] ? in[3 * col[t] + q] : R(0);
      }
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        a0 += v[t][0] * x[t][0] + v[t][1] * x[t][1] + v[t][2] * x[t][2];
        a1 += v[t][3] * x[t][0] + v[t][4] * x[t][1] + v[t][5] * x[t][2];
        a2 += v[t][6] * x[t][0] + v[t][7] * x[t][1] + v[t][8] * x[t][2];
      }
    }
#pragma unroll
    for (int o = kG / 2; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
      a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (has && gl < 3) {
      const int64_t d = 3 * r + gl;
      const R o = gl == 0 ? a0 : (gl == 1 ? a1 : a2);
      const R od = freem[d] ? o : R(0);
      out[d] = od;
      dot += (double)od * (double)w[d];
    }
  }
  return dot;
}

template <typename R>
struct PersistArgs {
  const int64_t* rowptr;
  const int32_t* cols;
  const R* vals;
  const uint8_t* freem;
  const R* minv;
  const double* b;
  double bscale, rtol2;
  R *x, *r, *z, *pa, *pb, *q;
  const R* x0;    // initial guess (zero on the fixed dofs), nullptr = 0
  int64_t n_nodes, maxit;
  int block3;
  PcgScalars* sc;
  double* part;   // 2 buffers x gridDim.x pairs
  unsigned long long spin_limit;   // bound of each grid-barrier wait (polls)
};

template <typename R>
__device__ __forceinline__ void precond_apply(const R* minv, int block3, int64_t n, const R rv[3], R zv[3]) {
  if (block3) {
    const R* M = minv + 9 * n;
#pragma unroll
    for (int i = 0; i < 3; ++i) zv[i] = M[3 * i] * rv[0] + M[3 * i + 1] * rv[1] + M[3 * i + 2] * rv[2];
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) zv[i] = minv[3 * n + i] * rv[i];
  }
}

// MINB = CTAs per SM the registers are budgeted for: 4 (64 registers) for FP32 blocks, 3 for
// FP64 blocks (two double blocks per lane in flight).  With the eight-lanes-per-row SpMV
// below, 4 is faster than 6 (40 registers, which spills) at every size measured, from the
// 222k-dof plate to 3.09M dofs.
template <typename R, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) pcg_persistent_kernel(const PersistArgs<R> a) {
  const int64_t n0 = (int64_t)blockIdx.x * a.n_nodes / gridDim.x;
  const int64_t n1 = (int64_t)(blockIdx.x + 1) * a.n_nodes / gridDim.x;
  PcgScalars* sc = a.sc;
  // publish this CTA's partial pair, then the fused barrier + reduction; the partial
  // buffers alternate, so a fast CTA never overwrites pairs a slow CTA may still be summing
  int red = 0;
  auto allreduce = [&](double v0, double v1, double& t0, double& t1) -> bool {
    block_sum2(v0, v1);
    double* pp = a.part + 2 * (size_t)gridDim.x * (red & 1);
    if (threadIdx.x == 0) {
      pp[2 * blockIdx.x] = v0;
      pp[2 * blockIdx.x + 1] = v1;
    }
    ++red;
    return grid_allreduce(&sc->gs, pp, t0, t1, a.spin_limit);
  };
  // x = x0 (or 0), r = b - K x0 on the free dofs, z = M^-1 r, p_prev = 0 (beta = 0 in the
  // first iteration); convergence is measured against |b|, as for a zero start
  if (a.x0 != nullptr) {
    spmv_range(a.rowptr, a.cols, a.vals, a.freem, a.x0, a.q, a.x0, n0, n1);
    __syncthreads();
  }
  double rz = 0.0, rr = 0.0, bb = 0.0, unused0 = 0.0;
  for (int64_t n = n0 + threadIdx.x; n < n1; n += kBlock) {
    R rv[3], zv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int64_t d = 3 * n + i;
      const R bd = a.freem[d] ? (R)(a.bscale * a.b[d]) : R(0);
      bb += (double)bd * (double)bd;
      rv[i] = a.x0 != nullptr ? bd - a.q[d] : bd;
      a.r[d] = rv[i];
      a.x[d] = a.x0 != nullptr ? a.x0[d] : R(0);
      a.pa[d] = R(0);
    }
    precond_apply(a.minv, a.block3, n, rv, zv);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      a.z[3 * n + i] = zv[i];
      rz += (double)rv[i] * (double)zv[i];
      rr += (double)rv[i] * (double)rv[i];
    }
  }
  if (!allreduce(rz, rr, rz, rr)) return;
  if (!allreduce(bb, 0.0, bb, unused0)) return;
  const double rr0 = bb;
  const double target = a.rtol2 * rr0;
  int breakdown = (isfinite(rz) && isfinite(rr) && isfinite(bb)) ? 0 : 1;
  int done = (!breakdown && rr <= target) ? 1 : 0;
  if (!breakdown && bb == 0.0) {   // b = 0: x = 0 whatever the initial guess
    for (int64_t d = 3 * n0 + threadIdx.x; d < 3 * n1; d += kBlock) a.x[d] = R(0);
    rr = 0.0;
    done = 1;
  }
  double beta = 0.0, pq = 0.0;
  int64_t it = 0;
  R* pprev = a.pa;
  R* pcur = a.pb;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  constexpr int kWarps = kBlock / 32;
  while (!done && !breakdown && it < a.maxit) {
    // q = K p with p = z + beta p_prev (rows without the Dirichlet columns: p is zero there),
    // eight lanes per block row as in spmv_range
    const R bt = (R)beta;
    double dot = 0.0;
    {
      constexpr int kG = 8;                  // lanes per block row
      constexpr int kRows = 32 / kG;         // block rows per warp and pass
      const int grp = lane / kG, gl = lane % kG;
      for (int64_t base = n0 + (int64_t)warp * kRows; base < n1; base += (int64_t)kWarps * kRows) {
        const int64_t r = base + grp;
        const bool has = r < n1;
        int64_t b = 0, e = 0;
        if (has) {
          b = a.rowptr[r];
          e = a.rowptr[r + 1];
        }
        R a0 = R(0), a1 = R(0), a2 = R(0);
        for (int64_t c = b; c < e; c += 2 * kG) {
          int64_t col[2];
          bool ok[2];
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const int64_t k = c + gl + t * kG;
            ok[t] = k < e;
            col[t] = ok[t] ? (int64_t)a.cols[k] : 0;
          }
          R v[2][9], x[2][3];
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const int64_t k = c + gl + t * kG;
#pragma unroll
            for (int q = 0; q < 9; ++q) v[t][q] = ok[t] ? a.vals[k * 9 + q] : R(0);
#pragma unroll
            for (int q = 0; q < 3; ++q)
              x[t][q] = ok[t] ? a.z[3 * col[t] + q] + bt * pprev[3 * col[t] + q] : R(0);
          }
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            a0 += v[t][0] * x[t][0] + v[t][1] * x[t][1] + v[t][2] * x[t][2];
            a1 += v[t][3] * x[t][0] + v[t][4] * x[t][1] + v[t][5] * x[t][2];
            a2 += v[t][6] * x[t][0] + v[t][7] * x[t][1] + v[t][8] * x[t][2];
          }
        }
#pragma unroll
        for (int o = kG / 2; o > 0; o >>= 1) {
          a0 += __shfl_xor_sync(0xffffffffu, a0, o);
          a1 += __shfl_xor_sync(0xffffffffu, a1, o);
          a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (has && gl < 3) {
          const int64_t d = 3 * r + gl;
          const R o = gl == 0 ? a0 : (gl == 1 ? a1 : a2);
          const R pd = a.z[d] + bt * pprev[d];
          const R qd = a.freem[d] ? o : R(0);
          pcur[d] = pd;
          a.q[d] = qd;
          dot += (double)pd * (double)qd;
        }
      }
    }
    double unused;
    if (!allreduce(dot, 0.0, pq, unused)) return;
    if (!(pq > 0.0) || !isfinite(pq)) {   // negative curvature or breakdown: x stays at the last iterate
      breakdown = 1;
      break;
    }
    const R al = (R)(rz / pq);
    // x += alpha p, r -= alpha q, z = M^-1 r on the own rows
    double rzn = 0.0, rrn = 0.0;
    for (int64_t n = n0 + threadIdx.x; n < n1; n += kBlock) {
      R rv[3], zv[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int64_t d = 3 * n + i;
        a.x[d] += al * pcur[d];
        rv[i] = a.r[d] - al * a.q[d];
        a.r[d] = rv[i];
      }
      precond_apply(a.minv, a.block3, n, rv, zv);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        a.z[3 * n + i] = zv[i];
        rzn += (double)rv[i] * (double)zv[i];
        rrn += (double)rv[i] * (double)rv[i];
      }
    }
    if (!allreduce(rzn, rrn, rzn, rrn)) return;
    ++it;
    if (!isfinite(rzn) || !isfinite(rrn)) { breakdown = 1; break; }
    beta = rz > 0.0 ? rzn / rz : 0.0;
    rz = rzn;
    rr = rrn;
    if (rr <= target) done = 1;
    R* tmp = pprev;
    pprev = pcur;
    pcur = tmp;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rz = rz;
    sc->rr = rr;
    sc->rr0 = rr0;
    sc->pq = pq;
    sc->target = target;
    sc->iters = (int)it;
    sc->breakdown = breakdown;
    sc->done = done;
  }
}


// ---------------------------------------------------------------------------------------
// One-launch CG with the streamed SpMV.  The iteration is that of pcg_persistent_kernel (same
// fixed-order reductions, the same two barriers) except for how q = K p is formed: the SpMV
// gathers z alone and q follows the recurrence q = K z + beta q_prev (K p = K z + beta K p_prev,
// the recurrence of Chronopoulos and Gear's CG), so each column costs one gathered vector
// instead of two; p = z + beta p_prev is formed on the own rows only.  The other change is how
// K reaches the SMs.  Each CTA owns a contiguous range of row chunks; a chunk's
// values and column indices are one contiguous range each in block-CSR order, and one thread
// brings them into shared memory with bulk asynchronous copies (cp.async.bulk, completion on
// an mbarrier), two stages deep, so that the HBM stream of K runs ahead of the arithmetic and
// arrives as whole 16-byte-aligned transfers.  The copy pipeline runs across iterations (K
// does not change during a solve): the copies of the next pass start while the current one
// finishes; the kernel drains the copies in flight before it exits.  Every wait is bounded.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bulk copy global -> shared of `bytes` (multiple of 16, both addresses 16-byte aligned),
// counted on the mbarrier's transaction count
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Bounded wait for phase `parity` of bar; false if the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned long long limit) {
  unsigned long long spins = 0;
  unsigned ns = 32;
  while (!mbar_try_wait(bar, parity)) {
    if (++spins > limit) return false;
    __nanosleep(ns);
    if (ns < 256) ns *= 2;
  }
  return true;
}

template <typename R>
struct StreamPipe {
  unsigned char* base;  // stage s at base + s * kStreamStageBytes
  uint64_t* bar;
  int64_t kc0;        // first chunk of this CTA
  int nck;            // chunks of this CTA
  long long seq;      // chunks consumed so far (across passes)
  long long issued;   // chunks issued so far
};

// Thread 0: start the copy of the CTA's chunk (issued mod nck) into stage (issued mod 2).
template <typename R>
__device__ __forceinline__ void stream_issue(StreamPipe<R>& sp, const int32_t* chunk, const int64_t* rowptr,
                                             const R* vals, const int32_t* cols) {
  const int st = (int)(sp.issued % kStreamStages);
  const int64_t c = sp.kc0 + (int64_t)(sp.issued % sp.nck);
  const int64_t b0 = rowptr[chunk[c]], b1 = rowptr[chunk[c + 1]];
  const uintptr_t v0 = (uintptr_t)(vals + 9 * b0), v1 = (uintptr_t)(vals + 9 * b1);
  const uintptr_t c0 = (uintptr_t)(cols + b0), c1 = (uintptr_t)(cols + b1);
  const uintptr_t va = v0 & ~(uintptr_t)15, vb = (v1 + 15) & ~(uintptr_t)15;
  const uintptr_t ca = c0 & ~(uintptr_t)15, cb = (c1 + 15) & ~(uintptr_t)15;
  const unsigned vbytes = (unsigned)(vb - va), cbytes = (unsigned)(cb - ca);
  uint64_t* bar = sp.bar + st;
  fence_proxy_async_smem();   // the stage's earlier contents were read through the generic proxy
  mbar_arrive_expect_tx(bar, vbytes + cbytes);
  unsigned char* dst = sp.base + (size_t)st * kStreamStageBytes;
  bulk_g2s(dst, (const void*)va, vbytes, bar);
  bulk_g2s(dst + stream_val_bytes<R>(), (const void*)ca, cbytes, bar);
  ++sp.issued;
}

// Thread 0, before the CTA exits: wait (bounded) for the copies still in flight.
template <typename R>
__device__ __forceinline__ void stream_drain(StreamPipe<R>& sp, unsigned long long limit) {
  for (long long k = sp.seq; k < sp.issued; ++k)
    mbar_wait(sp.bar + (int)(k % kStreamStages), (unsigned)((k / kStreamStages) & 1), limit);
}

template <typename R, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) pcg_stream_kernel(const PersistArgs<R> a, const int32_t* chunk,
                                                                  int64_t n_chunks) {
  extern __shared__ __align__(128) unsigned char s_stage[];
  __shared__ __align__(8) uint64_t s_bar[kStreamStages];
  __shared__ int s_fail;
  PcgScalars* sc = a.sc;
  StreamPipe<R> sp;
  sp.kc0 = (int64_t)blockIdx.x * n_chunks / gridDim.x;
  const int64_t kc1 = (int64_t)(blockIdx.x + 1) * n_chunks / gridDim.x;
  sp.nck = (int)(kc1 - sp.kc0);
  sp.bar = s_bar;
  sp.seq = 0;
  sp.issued = 0;
  sp.base = s_stage;
  const int64_t n0 = chunk[sp.kc0], n1 = chunk[kc1];
  if (threadIdx.x == 0) {
    s_fail = 0;
#pragma unroll
    for (int s2 = 0; s2 < kStreamStages; ++s2) mbar_init(&s_bar[s2], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // the first kStreamStages - 1 chunks of the first pass are on their way while the set-up
  // below runs
  if (threadIdx.x == 0 && sp.nck > 0)
    for (int k = 0; k < kStreamStages - 1; ++k) stream_issue<R>(sp, chunk, a.rowptr, a.vals, a.cols);

  int red = 0;
  auto allreduce = [&](double v0, double v1, double& t0, double& t1) -> bool {
    block_sum2(v0, v1);
    double* pp = a.part + 2 * (size_t)gridDim.x * (red & 1);
    if (threadIdx.x == 0) {
      pp[2 * blockIdx.x] = v0;
      pp[2 * blockIdx.x + 1] = v1;
    }
    ++red;
    return grid_allreduce(&sc->gs, pp, t0, t1, a.spin_limit);
  };
  bool alive = true;   // false once a wait has run out: skip to the drain
  if (a.x0 != nullptr) {
    spmv_range(a.rowptr, a.cols, a.vals, a.freem, a.x0, a.q, a.x0, n0, n1);
    __syncthreads();
  }
  double rz = 0.0, rr = 0.0, bb = 0.0, unused0 = 0.0;
  for (int64_t n = n0 + threadIdx.x; n < n1; n += kBlock) {
    R rv[3], zv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int64_t d = 3 * n + i;
      const R bd = a.freem[d] ? (R)(a.bscale * a.b[d]) : R(0);
      bb += (double)bd * (double)bd;
      rv[i] = a.x0 != nullptr ? bd - a.q[d] : bd;
      a.r[d] = rv[i];
      a.x[d] = a.x0 != nullptr ? a.x0[d] : R(0);
      a.pa[d] = R(0);
    }
    precond_apply(a.minv, a.block3, n, rv, zv);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      a.z[3 * n + i] = zv[i];
      rz += (double)rv[i] * (double)zv[i];
      rr += (double)rv[i] * (double)rv[i];
    }
  }
  double rr0 = 0.0, target = 0.0, beta = 0.0, pq = 0.0;
  int breakdown = 0, done = 0;
  int64_t it = 0;
  if (!allreduce(rz, rr, rz, rr) || !allreduce(bb, 0.0, bb, unused0)) alive = false;
  if (alive) {
    rr0 = bb;
    target = a.rtol2 * rr0;
    breakdown = (isfinite(rz) && isfinite(rr) && isfinite(bb)) ? 0 : 1;
    done = (!breakdown && rr <= target) ? 1 : 0;
    if (!breakdown && bb == 0.0) {   // b = 0: x = 0 whatever the initial guess
      for (int64_t d = 3 * n0 + threadIdx.x; d < 3 * n1; d += kBlock) a.x[d] = R(0);
      rr = 0.0;
      done = 1;
    }
  }
  R* pprev = a.pa;
  R* pcur = a.pb;
  constexpr int kL = stream_lanes<R>();          // lanes per row
  constexpr int kU = 32 / kL;                     // blocks per lane and round (32 per row and round)
  const int grp = threadIdx.x / kL, gl = threadIdx.x % kL;
  while (alive && !done && !breakdown && it < a.maxit) {
    const R bt = (R)beta;
    double dot = 0.0;
    for (int k = 0; k < sp.nck; ++k) {
      // chunk k is in stage seq mod kStreamStages; once every thread has seen it there and
      // is done with the previous chunk, that previous stage takes the copy of the chunk
      // kStreamStages - 1 ahead (wrapping into the next pass), so that kStreamStages - 1
      // copies run while this chunk is computed
      const int st = (int)(sp.seq % kStreamStages);
      const bool ok = mbar_wait(&s_bar[st], (unsigned)((sp.seq / kStreamStages) & 1), a.spin_limit);
      if (__syncthreads_or(!ok)) { alive = false; break; }
      if (threadIdx.x == 0) stream_issue<R>(sp, chunk, a.rowptr, a.vals, a.cols);
      const int64_t c = sp.kc0 + k;
      const int64_t r0 = chunk[c], r1 = chunk[c + 1];
      const int64_t cb0 = a.rowptr[r0];
      // the chunk's first value and column sit at these offsets of the stage (alignment slack)
      const unsigned char* stg = s_stage + (size_t)st * kStreamStageBytes;
      const R* sv = reinterpret_cast<const R*>(stg + (((uintptr_t)(a.vals + 9 * cb0)) & 15));
      const int32_t* scol =
          reinterpret_cast<const int32_t*>(stg + stream_val_bytes<R>() + (((uintptr_t)(a.cols + cb0)) & 15));
      // rows past the chunk's end take an empty range, so that every lane runs the shuffles
      const int64_t r = r0 + grp;
      const bool has = r < r1;
      const int64_t b = has ? a.rowptr[r] : 0, e = has ? a.rowptr[r + 1] : 0;
      R a0 = R(0), a1 = R(0), a2 = R(0);
      for (int64_t j0 = b; j0 < e; j0 += 32) {
        // all column reads, then all gathers of z, then the arithmetic
        int64_t col[kU];
        bool okj[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int64_t j = j0 + gl + u * kL;
          okj[u] = j < e;
          col[u] = okj[u] ? (int64_t)scol[j - cb0] : 0;
        }
        R x[kU][3];
#pragma unroll
        for (int u = 0; u < kU; ++u)
#pragma unroll
          for (int i = 0; i < 3; ++i)
            x[u][i] = okj[u] ? a.z[3 * col[u] + i] : R(0);
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          if (okj[u]) {
            const R* v = sv + 9 * (j0 + gl + u * kL - cb0);
            a0 += v[0] * x[u][0] + v[1] * x[u][1] + v[2] * x[u][2];
            a1 += v[3] * x[u][0] + v[4] * x[u][1] + v[5] * x[u][2];
            a2 += v[6] * x[u][0] + v[7] * x[u][1] + v[8] * x[u][2];
          }
        }
      }
#pragma unroll
      for (int o = kL / 2; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
      }
      if (has && gl < 3) {
        const int64_t d = 3 * r + gl;
        const R o = gl == 0 ? a0 : (gl == 1 ? a1 : a2);
        const R pd = a.z[d] + bt * pprev[d];
        const R qd = (a.freem[d] ? o : R(0)) + (it > 0 ? bt * a.q[d] : R(0));
        pcur[d] = pd;
        a.q[d] = qd;
        dot += (double)pd * (double)qd;
      }
      ++sp.seq;
    }
    if (!alive) break;
    double unused;
    if (!allreduce(dot, 0.0, pq, unused)) { alive = false; break; }
    if (!(pq > 0.0) || !isfinite(pq)) {   // negative curvature or breakdown: x stays at the last iterate
      breakdown = 1;
      break;
    }
    const R al = (R)(rz / pq);
    double rzn = 0.0, rrn = 0.0;
    for (int64_t n = n0 + threadIdx.x; n < n1; n += kBlock) {
      R rv[3], zv[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int64_t d = 3 * n + i;
        a.x[d] += al * pcur[d];
        rv[i] = a.r[d] - al * a.q[d];
        a.r[d] = rv[i];
      }
      precond_apply(a.minv, a.block3, n, rv, zv);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        a.z[3 * n + i] = zv[i];
        rzn += (double)rv[i] * (double)zv[i];
        rrn += (double)rv[i] * (double)rv[i];
      }
    }
    if (!allreduce(rzn, rrn, rzn, rrn)) { alive = false; break; }
    ++it;
    if (!isfinite(rzn) || !isfinite(rrn)) { breakdown = 1; break; }
    beta = rz > 0.0 ? rzn / rz : 0.0;
    rz = rzn;
    rr = rrn;
    if (rr <= target) done = 1;
    R* tmp = pprev;
    pprev = pcur;
    pcur = tmp;
  }
  if (threadIdx.x == 0) {
    stream_drain<R>(sp, a.spin_limit);
    if (!alive) atomicExch(&sc->gs.timeout, 1);
  }
  if (alive && blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rz = rz;
    sc->rr = rr;
    sc->rr0 = rr0;
    sc->pq = pq;
    sc->target = target;
    sc->iters = (int)it;
    sc->breakdown = breakdown;
    sc->done = done;
  }
}

// ---------------------------------------------------------------------------------------
// Persistent BiCGSTAB (van der Vorst 1992) with the same block-Jacobi preconditioner applied
// on the right, for Newton corrections whose tangent turned out indefinite (CG met p.Kp <= 0).
// Same row split, fixed-order reductions and fused barriers as the CG kernel: one plain
// barrier and four barrier-reductions per iteration.
constexpr int kBicgRestart = 200;       // iterations between true-residual restarts
constexpr int kBicgMaxRestarts = 1000;

template <typename R>
struct BicgArgs {
  const int64_t* rowptr;
  const int32_t* cols;
  const R* vals;
  const uint8_t* freem;
  const R* minv;
  const double* b;
  double bscale, rtol2;
  R *x, *r, *rh, *p, *v, *y, *s, *z, *t;
  int64_t n_nodes, maxit;
  int block3;
  PcgScalars* sc;
  double* part;
  unsigned long long spin_limit;   // bound of each grid-barrier wait (polls)
};

template <typename R>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 8 ? 3 : 4) bicgstab_persistent_kernel(const BicgArgs<R> a) {
  const int64_t n0 = (int64_t)blockIdx.x * a.n_nodes / gridDim.x;
  const int64_t n1 = (int64_t)(blockIdx.x + 1) * a.n_nodes / gridDim.x;
  PcgScalars* sc = a.sc;
  int red = 0;
  auto allreduce = [&](double v0, double v1, double& t0, double& t1) -> bool {
    block_sum2(v0, v1);
    double* pp = a.part + 2 * (size_t)gridDim.x * (red & 1);
    if (threadIdx.x == 0) {
      pp[2 * blockIdx.x] = v0;
      pp[2 * blockIdx.x + 1] = v1;
    }
    ++red;
    return grid_allreduce(&sc->gs, pp, t0, t1, a.spin_limit);
  };
  // x = 0, r = rh = b on the free dofs, p = v = 0
  double rr = 0.0, dummy = 0.0;
  for (int64_t d = 3 * n0 + threadIdx.x; d < 3 * n1; d += kBlock) {
    const R rv = a.freem[d] ? (R)(a.bscale * a.b[d]) : R(0);
    a.r[d] = rv;
    a.rh[d] = rv;
    a.x[d] = R(0);
    a.p[d] = R(0);
    a.v[d] = R(0);
    rr += (double)rv * (double)rv;
  }
  if (!allreduce(rr, 0.0, rr, dummy)) return;
  const double rr0 = rr, target = a.rtol2 * rr0;
  double rho = rr, rho_old = 1.0, alpha = 1.0, omega = 1.0, rv_ = 0.0;
  double rhh = rr;   // |rh|^2
  int breakdown = (isfinite(rr)) ? 0 : 1;
  int done = (!breakdown && rr <= target) ? 1 : 0;
  int64_t it = 0;
  int restarts = 0;
  while (!done && !breakdown && it < a.maxit) {
    const double beta = (rho / rho_old) * (alpha / omega);
    // p = r + beta (p - omega v), y = M^-1 p on the own nodes
    for (int64_t n = n0 + threadIdx.x; n < n1; n += kBlock) {
      R pv[3], yv[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int64_t d = 3 * n + i;
        pv[i] = a.r[d] + (R)beta * (a.p[d] - (R)omega * a.v[d]);
        a.p[d] = pv[i];
      }
      precond_apply(a.minv, a.block3, n, pv, yv);
#pragma unroll
      for (int i = 0; i < 3; ++i) a.y[3 * n + i] = yv[i];
    }
    if (!allreduce(0.0, 0.0, dummy, dummy)) return;   // y complete
    double d1 = spmv_range(a.rowptr, a.cols, a.vals, a.freem, a.y, a.v, a.rh, n0, n1);
    if (!allreduce(d1, 0.0, rv_, dummy)) return;
    if (rv_ == 0.0 || !isfinite(rv_)) { breakdown = 1; break; }        // rh . v
    alpha = rho / rv_;
    // x += alpha y, s = r - alpha v, z = M^-1 s
    double ss = 0.0;
    for (int64_t n = n0 + threadIdx.x; n < n1; n += kBlock) {
      R sv[3], zv[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int64_t d = 3 * n + i;
        a.x[d] += (R)alpha * a.y[d];
        sv[i] = a.r[d] - (R)alpha * a.v[d];
        a.s[d] = sv[i];
        ss += (double)sv[i] * (double)sv[i];
      }
      precond_apply(a.minv, a.block3, n, sv, zv);
#pragma unroll
      for (int i = 0; i < 3; ++i) a.z[3 * n + i] = zv[i];
    }
    if (!allreduce(ss, 0.0, ss, dummy)) return;
    ++it;
    if (!isfinite(ss)) { breakdown = 2; break; }
    if (ss <= target) { rr = ss; done = 1; break; }
    // t = K z; omega = (t.s) / (t.t)
    double ts = 0.0, tt = 0.0;
    {
      // t.s from the SpMV's dot, t.t in a second pass over the own rows
      ts = spmv_range(a.rowptr, a.cols, a.vals, a.freem, a.z, a.t, a.s, n0, n1);
      __syncthreads();
      for (int64_t d = 3 * n0 + threadIdx.x; d < 3 * n1; d += kBlock) tt += (double)a.t[d] * (double)a.t[d];
    }
    if (!allreduce(ts, tt, ts, tt)) return;
    if (!(tt > 0.0) || !isfinite(ts)) { breakdown = 3; break; }
    omega = ts / tt;
    // x += omega z, r = s - omega t; rho = rh.r, rr = r.r
    double rhr = 0.0;
    rr = 0.0;
    for (int64_t d = 3 * n0 + threadIdx.x; d < 3 * n1; d += kBlock) {
      a.x[d] += (R)omega * a.z[d];
      const R rv = a.s[d] - (R)omega * a.t[d];
      a.r[d] = rv;
      rhr += (double)a.rh[d] * (double)rv;
      rr += (double)rv * (double)rv;
    }
    if (!allreduce(rhr, rr, rhr, rr)) return;
    if (!isfinite(rr)) { breakdown = 4; break; }
    if (rr <= target) { done = 1; break; }
    // restart on (near) breakdown - rh nearly orthogonal to r, or omega = 0 - and every
    // kBicgRestart iterations: the true residual b - K x replaces the recurred one (which
    // drifts, above all in FP32) and becomes the new shadow residual
    const bool near = omega == 0.0 || fabs(rhr) <= 1e-10 * sqrt(rr * rhh);
    if (near || it % kBicgRestart == 0) {
      if (++restarts > kBicgMaxRestarts) { breakdown = 5; break; }
      spmv_range(a.rowptr, a.cols, a.vals, a.freem, a.x, a.v, a.x, n0, n1);   // v <- K x (scratch)
      __syncthreads();
      double rr2 = 0.0;
      for (int64_t d = 3 * n0 + threadIdx.x; d < 3 * n1; d += kBlock) {
        const R rv = a.freem[d] ? (R)(a.bscale * a.b[d]) - a.v[d] : R(0);
        a.r[d] = rv;
        a.rh[d] = rv;
        a.p[d] = R(0);
        a.v[d] = R(0);
        rr2 += (double)rv * (double)rv;
      }
      if (!allreduce(rr2, 0.0, rr, dummy)) return;
      if (!isfinite(rr)) { breakdown = 4; break; }
      if (rr <= target) { done = 1; break; }
      rhh = rr;
      rho = rr;
      rho_old = alpha = omega = 1.0;
      continue;
    }
    rho_old = rho;
    rho = rhr;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rr = rr;
    sc->rr0 = rr0;
    sc->target = target;
    sc->iters = (int)it;
    sc->breakdown = breakdown;
    sc->done = done;
  }
}

inline unsigned nblk(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }
inline unsigned rblk(int64_t n, int per) {   // grid of a reducing (grid-stride) kernel
  int64_t b = (n + per - 1) / per;
  if (b > kMaxRedBlocks) b = kMaxRedBlocks;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

template <typename R>
void spmv(const Csr& K, const R* vals, const uint8_t* freem, const R* x, R* y, PcgScalars* sc, double* part,
          cudaStream_t s) {
  spmv_kernel<R, true><<<rblk(K.n_nodes, kBlock / 32), kBlock, 0, s>>>(K.rowptr, K.cols, vals, freem, x, y, K.n_nodes,
                                                                 sc, part);
}

template <typename R>
void spmv_rows(const Csr& K, const R* vals, const uint8_t* freem, const R* x, R* y, cudaStream_t s) {
  spmv_kernel<R, false><<<rblk(K.n_nodes, kBlock / 32), kBlock, 0, s>>>(K.rowptr, K.cols, vals, freem, x, y,
                                                                         K.n_nodes, nullptr, nullptr);
}

template <typename R>
void predictor_rhs(const double* R_, const R* Kd, const double* f_ext, double dt, const uint8_t* freem, double* b,
                   int64_t n_dof, cudaStream_t s) {
  predictor_rhs_kernel<R><<<nblk(n_dof, kBlock), kBlock, 0, s>>>(R_, Kd, f_ext, dt, freem, b, n_dof);
}

template <typename R>
void pcg_init(const double* b, double bscale, const uint8_t* freem, PcgVecs<R>& v, int block3, int64_t n_nodes,
              PcgScalars* sc, double* part, cudaStream_t s) {
  pcg_init_kernel<R><<<rblk(n_nodes, kBlock), kBlock, 0, s>>>(b, freem, bscale, v.x, v.r, v.z, v.p, v.minv,
                                                              block3, n_nodes, sc, part);
}

template <typename R>
void pcg_iteration(const Csr& K, const R* vals, const uint8_t* freem, PcgVecs<R>& v, int block3, PcgScalars* sc,
                   double* part, cudaStream_t s) {
  spmv_kernel<R, false><<<rblk(K.n_nodes, kBlock / 32), kBlock, 0, s>>>(K.rowptr, K.cols, vals, freem, v.p, v.q,
                                                                 K.n_nodes, sc, part);
  pcg_update_kernel<R><<<rblk(K.n_nodes, kBlock), kBlock, 0, s>>>(v.x, v.r, v.z, v.p, v.q, v.minv, block3,
                                                                  K.n_nodes, sc, part);
  pcg_p_kernel<R><<<nblk(3 * K.n_nodes, kBlock), kBlock, 0, s>>>(v.p, v.z, 3 * K.n_nodes, sc);
}


template <typename R>
cudaError_t pcg_persistent(const Csr& K, const R* vals, const uint8_t* freem, PcgVecs<R>& v, int block3,
                           const double* b, double bscale, double rtol2, int64_t maxit, PcgScalars* sc,
                           double* part, int64_t part_slots, uint64_t spin_limit, cudaStream_t s, const R* x0) {
  constexpr int kMinb = sizeof(R) == 8 ? 3 : 4;   // FP64 blocks need the registers of 3 CTAs per SM
  // FP32 blocks are streamed; FP64 blocks are loaded directly (measured at 3.09M dofs: FP32
  // 0.311 ms per iteration streamed against 0.343 direct; FP64 1.61 against 1.18 ms, its
  // 402-block stages holding only half as many rows)
  const int32_t* chunk = sizeof(R) == 4 ? K.chunk32 : nullptr;
  const int64_t n_chunks = sizeof(R) == 4 ? K.n_chunk32 : 0;
  const bool streamed = chunk != nullptr && n_chunks > 0;
  const void* fn = streamed ? (const void*)pcg_stream_kernel<R, 3> : (const void*)pcg_persistent_kernel<R, kMinb>;
  const int cap = streamed ? 3 : kMinb;
  const size_t smem = streamed ? (size_t)kStreamStages * kStreamStageBytes : 0;
  int dev = 0, n_sm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && streamed) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, smem);
  if (e != cudaSuccess) return e;
  // every CTA must be resident (cooperative launch); at most cap per SM, and the partial
  // buffers hold 2 x 2 doubles per CTA
  int64_t grid = (int64_t)n_sm * (per_sm < cap ? per_sm : cap);
  if (grid > part_slots / 4) grid = part_slots / 4;
  const int64_t useful = streamed ? n_chunks : (K.n_nodes + kBlock / 8 - 1) / (kBlock / 8);
  if (grid > useful) grid = useful;   // streamed: every CTA owns at least one chunk
  if (grid < 1) grid = 1;
  PersistArgs<R> a{K.rowptr, K.cols, vals, freem, v.minv, b, bscale, rtol2, v.x, v.r, v.z, v.p, v.p2, v.q, x0,
                   K.n_nodes, maxit, block3, sc, part, (unsigned long long)spin_limit};
  if (streamed) {
    void* args[] = {&a, (void*)&chunk, (void*)&n_chunks};
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kBlock), args, smem, s);
  }
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kBlock), args, 0, s);
}


template <typename R>
cudaError_t bicgstab_persistent(const Csr& K, const R* vals, const uint8_t* freem, PcgVecs<R>& v, int block3,
                                const double* b, double bscale, double rtol2, int64_t maxit, PcgScalars* sc,
                                double* part, int64_t part_slots, uint64_t spin_limit, cudaStream_t s) {
  const void* fn = (const void*)bicgstab_persistent_kernel<R>;
  int dev = 0, n_sm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, 0);
  if (e != cudaSuccess) return e;
  int64_t grid = (int64_t)n_sm * (per_sm < 4 ? per_sm : 4);
  if (grid > part_slots / 4) grid = part_slots / 4;
  const int64_t useful = (K.n_nodes + kBlock / 8 - 1) / (kBlock / 8);   // an 8-lane group per row at least
  if (grid > useful) grid = useful;
  if (grid < 1) grid = 1;
  BicgArgs<R> a{K.rowptr, K.cols, vals, freem, v.minv, b, bscale, rtol2, v.x, v.r, v.rh, v.p, v.q, v.y, v.p2, v.z,
                v.t, K.n_nodes, maxit, block3, sc, part, (unsigned long long)spin_limit};
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kBlock), args, 0, s);
}

template <typename R>
void precond_setup(const Csr& K, const R* vals, const int64_t* diag_slot, const uint8_t* freem, R* minv,
                   int block3, int* bad, cudaStream_t s) {
  precond_kernel<R><<<nblk(K.n_nodes, 128), 128, 0, s>>>(vals, diag_slot, freem, minv, block3, K.n_nodes, bad);
}

void free_norm(const double* R_, const uint8_t* freem, int64_t n_dof, PcgScalars* sc, double* part,
               cudaStream_t s, double* out) {
  free_norm_kernel<<<rblk(n_dof, kBlock), kBlock, 0, s>>>(R_, freem, n_dof, sc, part, out);
}

template <typename R>
void add_update(double* u, const R* x, const uint8_t* freem, int64_t n_dof, cudaStream_t s, double c) {
  add_update_kernel<R><<<nblk(n_dof, kBlock), kBlock, 0, s>>>(u, x, freem, c, n_dof);
}

void set_dirichlet(double* u, const int64_t* dof, const double* val, double t, int64_t n_fixed, cudaStream_t s) {
  if (n_fixed > 0) set_dirichlet_kernel<<<nblk(n_fixed, kBlock), kBlock, 0, s>>>(u, dof, val, t, n_fixed);
}

void to_double(const float* a, double* b, int64_t n, cudaStream_t s) {
  convert_kernel<float, double><<<nblk(n, kBlock), kBlock, 0, s>>>(a, b, n);
}
void to_float(const double* a, float* b, int64_t n, cudaStream_t s) {
  convert_kernel<double, float><<<nblk(n, kBlock), kBlock, 0, s>>>(a, b, n);
}

template void spmv<float>(const Csr&, const float*, const uint8_t*, const float*, float*, PcgScalars*, double*,
                          cudaStream_t);
template void spmv<double>(const Csr&, const double*, const uint8_t*, const double*, double*, PcgScalars*, double*,
                           cudaStream_t);
template void spmv_rows<float>(const Csr&, const float*, const uint8_t*, const float*, float*, cudaStream_t);
template void spmv_rows<double>(const Csr&, const double*, const uint8_t*, const double*, double*, cudaStream_t);
template void predictor_rhs<float>(const double*, const float*, const double*, double, const uint8_t*, double*,
                                   int64_t, cudaStream_t);
template void predictor_rhs<double>(const double*, const double*, const double*, double, const uint8_t*, double*,
                                    int64_t, cudaStream_t);
template void pcg_init<float>(const double*, double, const uint8_t*, PcgVecs<float>&, int, int64_t, PcgScalars*,
                              double*, cudaStream_t);
template void pcg_init<double>(const double*, double, const uint8_t*, PcgVecs<double>&, int, int64_t, PcgScalars*,
                               double*, cudaStream_t);
template void pcg_iteration<float>(const Csr&, const float*, const uint8_t*, PcgVecs<float>&, int, PcgScalars*,
                                   double*, cudaStream_t);
template void pcg_iteration<double>(const Csr&, const double*, const uint8_t*, PcgVecs<double>&, int, PcgScalars*,
                                    double*, cudaStream_t);
template cudaError_t pcg_persistent<float>(const Csr&, const float*, const uint8_t*, PcgVecs<float>&, int,
                                            const double*, double, double, int64_t, PcgScalars*, double*, int64_t,
                                            uint64_t, cudaStream_t, const float*);
template cudaError_t pcg_persistent<double>(const Csr&, const double*, const uint8_t*, PcgVecs<double>&, int,
                                             const double*, double, double, int64_t, PcgScalars*, double*, int64_t,
                                             uint64_t, cudaStream_t, const double*);
template cudaError_t bicgstab_persistent<float>(const Csr&, const float*, const uint8_t*, PcgVecs<float>&, int,
                                                 const double*, double, double, int64_t, PcgScalars*, double*, int64_t,
                                                 uint64_t, cudaStream_t);
template cudaError_t bicgstab_persistent<double>(const Csr&, const double*, const uint8_t*, PcgVecs<double>&, int,
                                                  const double*, double, double, int64_t, PcgScalars*, double*,
                                                  int64_t, uint64_t, cudaStream_t);
template void precond_setup<float>(const Csr&, const float*, const int64_t*, const uint8_t*, float*, int, int*,
                                   cudaStream_t);
template void precond_setup<double>(const Csr&, const double*, const int64_t*, const uint8_t*, double*, int, int*,
                                    cudaStream_t);
template void add_update<float>(double*, const float*, const uint8_t*, int64_t, cudaStream_t, double);
template void add_update<double>(double*, const double*, const uint8_t*, int64_t, cudaStream_t, double);

}  // namespace hfe
