// Small dense FP64 linear algebra on the device for the Davidson subspace
// (the O_ij = <psi_i|O|psi_j> matrices and their "subspace diagonalization",
// Sec. "New parallelization levels"):
//
//  * jacobi_eigh   Hermitian eigensolver, cyclic parallel (round-robin pairing)
//                  two-sided Jacobi with complex rotations; one cooperative
//                  launch, rounds separated by a bounded grid barrier.
//  * cholqr_factor Cholesky of a Gram matrix with column dropping, returning the
//                  k x k' transform Tr with T Tr orthonormal.
//  * hermitize     completes and symmetrises freshly computed columns of the
//                  subspace matrix.
//
// Every spin in these kernels is bounded (about one second of %globaltimer);
// a kernel that gives up records PWH_ERR_TIMEOUT in the device error word and
// returns.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "dense.cuh"
#include "gemm.cuh"

namespace pwh {

constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ uint64_t gtimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sense-counting grid barrier for a cooperative launch (all blocks resident).
// Returns false (after recording the error) if the wait ran out or another
// block already gave up.
struct GridBar {
  unsigned* count;
  unsigned* gen;
  int* abort;
  int* err;
};

__device__ bool grid_sync(const GridBar& gb) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = gb.gen;
    volatile int* vab = gb.abort;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(gb.count, 1u) == gridDim.x - 1) {
      *gb.count = 0;
      __threadfence();
      atomicAdd(gb.gen, 1u);
    } else {
      const uint64_t t0 = gtimer_ns();
      unsigned it = 0;
      while (*vgen == g) {
        if (*vab) { ok = 0; break; }
        if ((++it & 255) == 0 && gtimer_ns() - t0 > kWaitNs) {
          ok = 0;
          atomicExch(gb.abort, 1);
          atomicExch(gb.err, (int)PWH_ERR_TIMEOUT);
          break;
        }
      }
    }
    __threadfence();
    if (*vab) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Index at tournament position j in round r of a round-robin over n (even)
// players: position 0 fixed, the others rotate.
__device__ __forceinline__ int rr_player(int j, int r, int n) {
  return j == 0 ? 0 : 1 + ((j - 1 + r) % (n - 1));
}

__device__ __forceinline__ double cabs2(double2 z) { return z.x * z.x + z.y * z.y; }

// Parallel cyclic Jacobi on A (n x n Hermitian, column-major ld = n; ping-pong
// buffers A[0]/A[1], Q[0]/Q[1]; A[0] and Q[0] hold the start, Q[0] being the
// basis the start is expressed in).  n is padded to even np with a dummy index
// that never rotates.  In each round of the round-robin every pair (p, q)
// gets the rotation J = [[c, s e^{i phi}], [-s e^{-i phi}, c]] that zeroes
// A_pq; the np/2 rotations are disjoint, so A' = J^H A J and Q' = Q J are
// formed element-wise in one pass.  Every block recomputes all rotations of
// the round in shared memory from A's diagonal and upper pairs (cheap), so a
// round needs a single grid barrier, and every block sees the same largest
// |A_pq| of the sweep: the sweep loop stops in lockstep once it is
// <= tol * max|A_ii|.
struct JacobiArgs {
  double2* A[2];
  double2* Q[2];
  int n, np, max_sweeps;
  double tol;
  int* out_buf;   // buffer index (0/1) holding the result, sweeps used
  GridBar gb;
};

__global__ void k_jacobi(JacobiArgs a) {
  extern __shared__ __align__(16) unsigned char jsm[];
  const int n = a.n, np = a.np;
  // 16-byte entries first so that every table is naturally aligned for any np
  double2* jpart = (double2*)jsm;                    // np: J[partner(x)][x]
  double* jself = (double*)(jpart + np);             // np: J[x][x]
  int* partner = (int*)(jself + np);                 // np
  __shared__ double s_off[32], s_dmax[32];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  int cur = 0;
  int sweep = 0;
  for (; sweep < a.max_sweeps; ++sweep) {
    double sweep_off = 0.0, dmax = 0.0;
    for (int r = 0; r < np - 1; ++r) {
      const double2* A = a.A[cur];
      double off = 0.0, dm = 0.0;
      for (int i = threadIdx.x; i < np / 2; i += blockDim.x) {
        int p = rr_player(i, r, np), q = rr_player(np - 1 - i, r, np);
        if (p > q) { int t = p; p = q; q = t; }
        double c = 1.0, sr = 0.0, si = 0.0;
        if (q < n) {
          const double2 apq = A[(size_t)q * n + p];
          const double g = sqrt(cabs2(apq));
          const double app = A[(size_t)p * n + p].x, aqq = A[(size_t)q * n + q].x;
          dm = fmax(dm, fmax(fabs(app), fabs(aqq)));
          if (g > 0.0) {
            off = fmax(off, g);
            const double zeta = (aqq - app) / (2.0 * g);
            const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            c = 1.0 / sqrt(1.0 + t * t);
            const double sn = t * c;
            sr = sn * apq.x / g;
            si = sn * apq.y / g;
          }
        } else if (p < n) {
          dm = fmax(dm, fabs(A[(size_t)p * n + p].x));
        }
        partner[p] = q;
        partner[q] = p;
        jself[p] = c;
        jself[q] = c;
        jpart[p] = make_double2(-sr, si);  // J[q][p] = -s e^{-i phi}
        jpart[q] = make_double2(sr, si);   // J[p][q] =  s e^{+i phi}
      }
      for (int o = 16; o > 0; o >>= 1) {
        off = fmax(off, __shfl_xor_sync(0xffffffffu, off, o));
        dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
      }
      if ((threadIdx.x & 31) == 0) {
        s_off[threadIdx.x >> 5] = off;
        s_dmax[threadIdx.x >> 5] = dm;
      }
      __syncthreads();
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        sweep_off = fmax(sweep_off, s_off[w]);
        dm = fmax(dm, s_dmax[w]);
      }
      dmax = dm;
      const double2* Qc = a.Q[cur];
      double2* An = a.A[cur ^ 1];
      double2* Qn = a.Q[cur ^ 1];
      const int nn = n * n;
      for (int t = tid; t < 2 * nn; t += nth) {
        const bool isq = t >= nn;
        const int e = isq ? t - nn : t;
        const int i = e % n, j = e / n;
        const int pj = partner[j];
        const double cj = jself[j];
        const double2 jpj = jpart[j];
        if (!isq) {
          const int pi = partner[i];
          const double ci = jself[i];
          const double2 jpi = jpart[i];
          // (A J)[x][j] = A[x][j] J_jj + A[x][pj] J_pj,j ; A' = J^H (A J)
          double2 aij = scl<double>(A[(size_t)j * n + i], cj);
          if (pj < n) aij = add<double>(aij, mul<double>(A[(size_t)pj * n + i], jpj));
          double2 v = scl<double>(aij, ci);
          if (pi < n) {
            double2 apj = scl<double>(A[(size_t)j * n + pi], cj);
            if (pj < n) apj = add<double>(apj, mul<double>(A[(size_t)pj * n + pi], jpj));
            v = add<double>(v, mul<double>(make_double2(jpi.x, -jpi.y), apj));
          }
          An[(size_t)j * n + i] = v;
        } else {
          double2 v = scl<double>(Qc[(size_t)j * n + i], cj);
          if (pj < n) v = add<double>(v, mul<double>(Qc[(size_t)pj * n + i], jpj));
          Qn[(size_t)j * n + i] = v;
        }
      }
      cur ^= 1;
      if (!grid_sync(a.gb)) return;
    }
    if (sweep_off <= a.tol * fmax(dmax, 1e-300)) {
      ++sweep;
      break;
    }
  }
  if (tid == 0) {
    a.out_buf[0] = cur;
    a.out_buf[1] = sweep;
  }
}

// Sort the diagonal ascending and gather the lowest nk eigenpairs:
// theta[k], C[:, k] (n x nk, ld = n).  Also keeps the full eigenvector matrix
// in Qkeep (ld = ldk) for a warm start of the next call.  One block.
__global__ void k_jacobi_select(const double2* __restrict__ A0, const double2* __restrict__ A1,
                                const double2* __restrict__ Q0, const double2* __restrict__ Q1,
                                const int* __restrict__ buf, int n, int nk,
                                double* __restrict__ theta, double2* __restrict__ C,
                                double2* __restrict__ Qkeep, int64_t ldk) {
  const double2* A = buf[0] ? A1 : A0;
  const double2* Q = buf[0] ? Q1 : Q0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double di = A[(size_t)i * n + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double dj = A[(size_t)j * n + j].x;
      rank += (dj < di) || (dj == di && j < i);
    }
    if (rank < nk) {
      theta[rank] = di;
      for (int r = 0; r < n; ++r) C[(size_t)rank * n + r] = Q[(size_t)i * n + r];
    }
    if (Qkeep)
      for (int r = 0; r < n; ++r) Qkeep[(size_t)rank * ldk + r] = Q[(size_t)i * n + r];
  }
}

// Q0 = blockdiag(Qprev[0:m0, 0:m0], I) (n x n, ld n).
__global__ void k_warm_basis(const double2* __restrict__ Qprev, int64_t ldp, int m0, int n,
                             double2* __restrict__ Q0) {
  int64_t tot = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t % n), j = (int)(t / n);
    double2 v = make_double2(i == j ? 1.0 : 0.0, 0.0);
    if (i < m0 && j < m0) v = Qprev[(size_t)j * ldp + i];
    else if (i < m0 || j < m0) v = make_double2(0.0, 0.0);
    Q0[t] = v;
  }
}

// Complete columns [m0, m) of the Hermitian subspace matrix H (ld): rows
// [0, m0) mirror into the lower-left block; the new diagonal block is
// replaced by its Hermitian part.
__global__ void k_hermitize(double2* __restrict__ H, int64_t ld, int m0, int m) {
  const int k = m - m0;
  int64_t tot = (int64_t)m * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t % m), j = m0 + (int)(t / m);
    if (i < m0) {
      double2 z = H[(size_t)j * ld + i];
      H[(size_t)i * ld + j] = make_double2(z.x, -z.y);
    } else if (i < j) {
      double2 a = H[(size_t)j * ld + i], b = H[(size_t)i * ld + j];
      double2 av = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
      H[(size_t)j * ld + i] = av;
      H[(size_t)i * ld + j] = make_double2(av.x, -av.y);
    } else if (i == j) {
      H[(size_t)j * ld + i].y = 0.0;
    }
  }
}

// Cholesky-QR factor of a Gram matrix S = T^H T (k x k, ld = k), one block.
// Column j survives when S_jj > 0, sqrt(S_jj) >= drop_rel * t0[j] (t0 may be
// null) and its Cholesky pivot of the unit-diagonal matrix stays above
// piv_tol.  Output: Tr (k x k, ld = k) whose first kk columns give T Tr with
// orthonormal columns (other columns zero); *kk = number kept.  W: k x k
// scratch.
__global__ void k_cholqr(const double2* __restrict__ S, int k, const double* __restrict__ t0,
                         double drop_rel, double piv_tol, double2* __restrict__ W,
                         double2* __restrict__ Tr, int* __restrict__ kk) {
  __shared__ int keep_s[1024];
  __shared__ int rank_s[1024];
  __shared__ double dinv_s[1024];
  __shared__ int nkeep_s;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double d = S[(size_t)j * k + j].x;
    bool keep = d > 0.0 && (!t0 || sqrt(d) >= drop_rel * t0[j]);
    keep_s[j] = keep;
    dinv_s[j] = keep ? 1.0 / sqrt(d) : 0.0;
  }
  __syncthreads();
  // W = D^-1/2 S D^-1/2
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    int i = t % k, j = t / k;
    W[t] = scl<double>(S[t], dinv_s[i] * dinv_s[j]);
  }
  __syncthreads();
  // right-looking Cholesky on the kept set (lower triangle of W becomes L)
  for (int j = 0; j < k; ++j) {
    __shared__ double piv_s;
    if (threadIdx.x == 0) {
      double piv = W[(size_t)j * k + j].x;
      if (keep_s[j] && !(piv > piv_tol)) keep_s[j] = 0;
      piv_s = keep_s[j] ? sqrt(piv) : 0.0;
    }
    __syncthreads();
    if (keep_s[j]) {
      const double lj = piv_s;
      for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x)
        if (keep_s[i]) W[(size_t)j * k + i] = scl<double>(W[(size_t)j * k + i], 1.0 / lj);
      __syncthreads();
      // A_il -= L_ij conj(L_lj) for kept i >= l > j
      for (int t = threadIdx.x; t < (k - j - 1) * (k - j - 1); t += blockDim.x) {
        int i = j + 1 + t % (k - j - 1), l = j + 1 + t / (k - j - 1);
        if (i >= l && keep_s[i] && keep_s[l]) {
          double2 lij = W[(size_t)j * k + i], llj = W[(size_t)j * k + l];
          W[(size_t)l * k + i] = sub<double>(W[(size_t)l * k + i], mulc<double>(lij, llj));
        }
      }
      if (threadIdx.x == 0) W[(size_t)j * k + j] = make_double2(lj, 0.0);
    }
    __syncthreads();
  }
  // compress kept indices
  if (threadIdx.x == 0) {
    int c = 0;
    for (int j = 0; j < k; ++j) rank_s[j] = keep_s[j] ? c++ : -1;
    nkeep_s = c;
    *kk = c;
  }
  __syncthreads();
  const int kp = nkeep_s;
  // Tr = D^-1/2 L^-H: column c of Tr (c < kp) is D^-1/2 times row c of L^-1
  // conjugated; solve L^H x = e_c by back substitution over kept indices.
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) Tr[t] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    if (!keep_s[j]) continue;
    const int c = rank_s[j];
    // x = L^-H e_c (upper triangular solve): x_i for kept i <= j (in rank order)
    // Use Tr column c as storage (rows = original indices).
    double2* x = Tr + (size_t)c * k;
    for (int i = j; i >= 0; --i) {
      if (!keep_s[i]) continue;
      double2 v = make_double2(i == j ? 1.0 : 0.0, 0.0);
      for (int l = i + 1; l <= j; ++l)
        if (keep_s[l]) {
          // (L^H)_{il} = conj(L_li)
          double2 lli = W[(size_t)i * k + l];
          v = sub<double>(v, mul<double>(make_double2(lli.x, -lli.y), x[l]));
        }
      x[i] = scl<double>(v, 1.0 / W[(size_t)i * k + i].x);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < k * kp; t += blockDim.x) {
    int i = t % k;
    Tr[t] = scl<double>(Tr[t], dinv_s[i]);
  }
}

// ---------------------------------------------------------------- host -----
void jacobi_eigh(System& s, DenseWs& w, const double2* H, int64_t ldh, int n, int nk,
                 double* theta, double2* C, cudaStream_t st, double2* Qkeep, int64_t ldk,
                 int warm_m0) {
  if (n > kJacobiMaxN) throw Error{PWH_ERR_ARG, "subspace larger than the Jacobi limit"};
  const int np = n + (n & 1);
  const size_t nn = (size_t)n * n;
  ensure(w.jac, 4 * nn * sizeof(double2) + 64);
  double2* A0 = (double2*)w.jac.p;
  double2* A1 = A0 + nn;
  double2* Q0 = A1 + nn;
  double2* Q1 = Q0 + nn;
  if (!w.ctl) PWH_CUDA(cudaMalloc((void**)&w.ctl, 64));
  unsigned* ctl = (unsigned*)w.ctl;
  PWH_CUDA(cudaMemsetAsync(ctl, 0, 64, st));
  const int gq = (int)std::min<int64_t>(1024, ((int64_t)nn + 255) / 256);
  if (warm_m0 > 0 && Qkeep) {
    // start from the previous eigenbasis: A = Q0^H H Q0, Q = Q0
    k_warm_basis<<<gq, 256, 0, st>>>(Qkeep, ldk, warm_m0, n, Q0);
    PWH_LAUNCH_CHECK();
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
    cgemm<double>(s, false, n, n, n, one, H, ldh, Q0, n, zero, A1, n, st);
    cgemm<double>(s, true, n, n, n, one, Q0, n, A1, n, zero, A0, n, st);
    hermitize(A0, n, 0, n, st);
  } else {
    PWH_CUDA(cudaMemcpy2DAsync(A0, n * sizeof(double2), H, ldh * sizeof(double2),
                               n * sizeof(double2), n, cudaMemcpyDeviceToDevice, st));
    k_warm_basis<<<gq, 256, 0, st>>>(nullptr, 0, 0, n, Q0);
    PWH_LAUNCH_CHECK();
  }
  JacobiArgs a;
  a.A[0] = A0; a.A[1] = A1; a.Q[0] = Q0; a.Q[1] = Q1;
  a.n = n; a.np = np; a.max_sweeps = 40; a.tol = 1e-13;
  a.out_buf = (int*)(ctl + 8);
  a.gb.count = ctl; a.gb.gen = ctl + 1; a.gb.abort = (int*)(ctl + 2);
  a.gb.err = device_error_word(s);
  const size_t smem = (size_t)(np + 2) * sizeof(int) + (size_t)np * (sizeof(double) + sizeof(double2)) + 16;
  static bool attr = false;
  if (!attr) {
    PWH_CUDA(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  int dev = 0, nsm = 0, per_sm = 0;
  PWH_CUDA(cudaGetDevice(&dev));
  PWH_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  PWH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, 256, smem));
  const int want = (int)std::max<int64_t>(1, std::min<int64_t>((2 * (int64_t)nn + 1023) / 1024, nsm));
  const int blocks = std::max(1, std::min(want, nsm * std::max(per_sm, 1)));
  void* args[] = {&a};
  {
    // work recorded after the launch, once the number of sweeps is known
    TimedScope ts(s, KF_JACOBI, st);
    PWH_CUDA(cudaLaunchCooperativeKernel((void*)k_jacobi, blocks, 256, args, smem, st));
    note_launch();
  }
  k_jacobi_select<<<1, 256, 0, st>>>(A0, A1, Q0, Q1, a.out_buf, n, nk, theta, C, Qkeep, ldk);
  PWH_LAUNCH_CHECK();
}

void hermitize(double2* H, int64_t ld, int m0, int m, cudaStream_t st) {
  if (m <= m0) return;
  int64_t tot = (int64_t)m * (m - m0);
  int blocks = (int)std::min<int64_t>(1024, (tot + 255) / 256);
  k_hermitize<<<blocks, 256, 0, st>>>(H, ld, m0, m);
  PWH_LAUNCH_CHECK();
}

void cholqr_factor(System& s, DenseWs& w, const double2* S, int k, const double* t0,
                   double drop_rel, double2* Tr, int* kk, cudaStream_t st) {
  if (k > 1024) throw Error{PWH_ERR_ARG, "block of more than 1024 new directions"};
  ensure(w.chol, (size_t)k * k * sizeof(double2));
  TimedScope ts(s, KF_CHOLQR, st);
  k_cholqr<<<1, 1024, 0, st>>>(S, k, t0, drop_rel, 1e-12, (double2*)w.chol.p, Tr, kk);
  PWH_LAUNCH_CHECK();
}

}  // namespace pwh
