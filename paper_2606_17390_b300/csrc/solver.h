// Solver kernels of the Newton step (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace hfe {

constexpr int kMaxRedBlocks = 148 * 16;   // grid cap of the reducing kernels (grid-stride)

struct Csr {            // block-CSR pattern of K over node pairs (3x3 blocks)
  const int64_t* rowptr;
  const int32_t* cols;
  int64_t n_nodes;
  int64_t n_blocks;
  // row chunks of the streamed SpMV of the one-launch CG, for FP32 and FP64 values: chunk c is
  // rows [chunk[c], chunk[c+1]) (at most kStreamRows rows and stream_max_blocks<R>() blocks);
  // nullptr / 0 when the pattern has a row too long for a chunk (the CG then loads directly)
  const int32_t* chunk32 = nullptr;
  int64_t n_chunk32 = 0;
  const int32_t* chunk64 = nullptr;
  int64_t n_chunk64 = 0;
};

// Streamed SpMV: each CTA of the one-launch CG copies its chunks of K (values and column
// indices, contiguous in block-CSR order) into shared memory with bulk asynchronous copies,
// two stages deep.  kStreamStageBytes bounds one stage; a chunk holds at most
// stream_rows<R>() rows: one row per group of stream_lanes<R>() lanes of the 256-thread CTA.
template <typename R>
__host__ __device__ constexpr int stream_lanes() { return sizeof(R) == 4 ? 8 : 16; }
template <typename R>
__host__ __device__ constexpr int stream_rows() { return 256 / stream_lanes<R>(); }
constexpr int kStreamStages = 2;
constexpr int kStreamStageBytes = 30 * 1024;
// values (9 R per block) and columns (4 B per block) of a chunk, each with up to 16 B of
// alignment slack at its start and rounded up to 16 B at its end
template <typename R>
__host__ __device__ constexpr int stream_max_blocks() {
  return (kStreamStageBytes - 128) / (9 * (int)sizeof(R) + 4);
}
// a copy of n bytes starting anywhere covers at most n + 30 bytes once both ends are rounded
template <typename R>
__host__ __device__ constexpr int stream_val_bytes() {
  return ((stream_max_blocks<R>() * 9 * (int)sizeof(R) + 32 + 15) / 16) * 16;
}
template <typename R>
__host__ __device__ constexpr int stream_col_bytes() {
  return ((stream_max_blocks<R>() * 4 + 32 + 15) / 16) * 16;
}
static_assert(stream_val_bytes<float>() + stream_col_bytes<float>() <= kStreamStageBytes, "stage");
static_assert(stream_val_bytes<double>() + stream_col_bytes<double>() <= kStreamStageBytes, "stage");
// Elements of padding past the end of every K value and column array: the bulk copies round
// their end up to 16 bytes.
constexpr int kKPad = 16;
// stream_chunks (the host-side cut of the rows into chunks) is declared in pattern.h.

// Grid-barrier words of the persistent solver, each in its own 128-byte line so that the
// CTAs polling the generation do not contend with the arrivals.
struct __align__(128) GridSync {
  unsigned count;       // CTAs arrived at the current barrier
  unsigned pad0[31];
  unsigned gen;         // barrier generation, bumped by the last arrival
  unsigned pad1[31];
  int timeout;          // a barrier wait ran out (never expected; the solve stops)
  int pad2[31];
  double tot[2];        // the reduction the last arrival computed for everyone
  double pad3[14];
};

struct PcgScalars {     // device-resident CG scalars
  double rz, rr, rr0, pq, alpha, beta, norm2, nonfinite;
  double target;        // rr at which the solve has converged (set by the host)
  unsigned ticket;
  int breakdown;
  int iters;
  int done;             // set once rr <= target: later iterations leave x unchanged
  GridSync gs;          // persistent solver only
};

template <typename R>
struct PcgVecs {
  R *x, *r, *z, *p, *q, *minv;
  R* p2;                // second search-direction buffer of the persistent solver
  R *rh, *y, *t;        // BiCGSTAB: shadow residual, preconditioned direction, K z
};

inline int64_t partial_slots() { return 2 * (int64_t)kMaxRedBlocks; }

template <typename R>
void spmv(const Csr& K, const R* vals, const uint8_t* freem, const R* x, R* y, PcgScalars* sc, double* part,
          cudaStream_t s);
// y = K x over all columns (no Dirichlet elimination), fixed rows set to 0
template <typename R>
void spmv_rows(const Csr& K, const R* vals, const uint8_t* freem, const R* x, R* y, cudaStream_t s);
template <typename R>
void predictor_rhs(const double* R_, const R* Kd, const double* f_ext, double dt, const uint8_t* freem, double* b,
                   int64_t n_dof, cudaStream_t s);
template <typename R>
void pcg_init(const double* b, double bscale, const uint8_t* freem, PcgVecs<R>& v, int block3, int64_t n_nodes,
              PcgScalars* sc, double* part, cudaStream_t s);
template <typename R>
void pcg_iteration(const Csr& K, const R* vals, const uint8_t* freem, PcgVecs<R>& v, int block3, PcgScalars* sc,
                   double* part, cudaStream_t s);
// Whole PCG solve in one cooperative launch (grid barriers, no host round trips): x = K^-1 b
// to |r| <= sqrt(rtol2) |b| or maxit iterations, from x0 (nullptr = 0; must not alias v's
// vectors); results in *sc (iters, rr, rr0 = |b|^2, rz, pq, breakdown, done, gs.timeout).
// *sc must be zeroed before the launch.
// spin_limit bounds every grid-barrier wait (polls); a wait that runs out sets sc->gs.timeout.
template <typename R>
cudaError_t pcg_persistent(const Csr& K, const R* vals, const uint8_t* freem, PcgVecs<R>& v, int block3,
                           const double* b, double bscale, double rtol2, int64_t maxit, PcgScalars* sc,
                           double* part, int64_t part_slots, uint64_t spin_limit, cudaStream_t s,
                           const R* x0 = nullptr);
// Preconditioned BiCGSTAB in one cooperative launch for a symmetric indefinite (or
// nonsymmetric) K with the same SPD block-Jacobi preconditioner: x (v.x) = K^-1 b; uses v.r,
// v.rh, v.p, v.q (as v), v.y, v.p2 (as s), v.z, v.t.  Results in *sc as for pcg_persistent.
template <typename R>
cudaError_t bicgstab_persistent(const Csr& K, const R* vals, const uint8_t* freem, PcgVecs<R>& v, int block3,
                                const double* b, double bscale, double rtol2, int64_t maxit, PcgScalars* sc,
                                double* part, int64_t part_slots, uint64_t spin_limit, cudaStream_t s);
template <typename R>
void precond_setup(const Csr& K, const R* vals, const int64_t* diag_slot, const uint8_t* freem, R* minv,
                   int block3, int* bad, cudaStream_t s);
// ||R_free||^2 into sc->norm2 and, if out != nullptr, ||R_free|| into *out (device)
void free_norm(const double* R_, const uint8_t* freem, int64_t n_dof, PcgScalars* sc, double* part,
               cudaStream_t s, double* out);
// u += c x on the free dofs
template <typename R>
void add_update(double* u, const R* x, const uint8_t* freem, int64_t n_dof, cudaStream_t s, double c = 1.0);
void set_dirichlet(double* u, const int64_t* dof, const double* val, double t, int64_t n_fixed, cudaStream_t s);
void to_double(const float* a, double* b, int64_t n, cudaStream_t s);
void to_float(const double* a, float* b, int64_t n, cudaStream_t s);

}  // namespace hfe
