// FP32 parallel cyclic Jacobi with the whole matrix resident in the shared
// memory of one thread-block cluster (16 CTAs on one GPC), for the subspace
// diagonalisation of the block Davidson method (Sec. "New parallelization
// levels": the O_ij = <psi_i|O|psi_j> matrices and their diagonalization).
//
// The same two-sided complex Jacobi as k_jacobi (round-robin pairing, np - 1
// rounds a sweep, every round rotates np/2 disjoint pairs), distributed by
// column pairs instead of through global memory:
//
//  * tournament positions 0..np-1: pair k plays positions k and np-1-k; CTA c
//    owns pairs [c PP, c PP + PP) and keeps, for each of its positions, the
//    full column of A and of Q (rows in original index order) of the index
//    ("player") standing there.  Between rounds every player except the one
//    at position 0 steps to the next position (np-1 wraps to 1); only the
//    players crossing to a neighbouring CTA move data (at most two columns of
//    A and two of Q per CTA and round, written into the neighbour's inbox
//    through distributed shared memory), the rest move by table update.
//  * a round: each CTA computes the rotations of its own pairs and publishes
//    them, cluster barrier, each CTA reads all np/2 rotations, then applies
//    J^H A J to its own columns (2 x 2 blocks: row pair x own column pair, in
//    place) and Q J to its own Q columns; the crossing columns go to the
//    inboxes, cluster barrier, inbox columns land in the freed buffers.
//  * after each sweep every CTA publishes max |A_ij| (i != j) and max |A_ii|
//    of its columns; all CTAs take the same decision from the same numbers,
//    so the control flow stays uniform and every barrier is met.
//
// No software spin anywhere: only the hardware cluster barrier.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "dense.cuh"
#include "jacobi_rot.cuh"

namespace cg = cooperative_groups;

namespace pwh {

constexpr int kDsmCluster = 16;
constexpr int kDsmThreads = 1024;

struct JdsmArgs {
  const double2* A;  // n x n Hermitian start (full), ld lda
  int64_t lda;
  double2* Q;        // out: eigenvectors, column j for index j, ld ldq
  int64_t ldq;
  double* diag;      // out: final diagonal (eigenvalue estimates), n
  int* info;         // out: [0] = 0, [1] = sweeps used
  int n, np, P, PP, max_sweeps;
  float tol;
};

// shared-memory layout of one CTA (element counts), in this order:
//   float2 colA[nbuf n], colQ[nbuf n], alls[P], rs[PP]
//   float  allc[P], rc[PP], red[2 + 64]
//   int    allp[P], allq[P], rp[PP], rq[PP], rbp[PP], rbq[PP],
//          tab[4][2 PP] (player/buffer, current and next), misc[16]
// with nbuf = 2 PP + 2 (two inbox buffers at the end).
__host__ __device__ inline size_t jdsm_smem_bytes(int n, int P, int PP) {
  const size_t nbuf = 2 * (size_t)PP + 2;
  return (2 * nbuf * n + P + PP) * sizeof(float2) + (size_t)(P + PP + 66) * sizeof(float) +
         (size_t)(2 * P + 4 * PP + 8 * PP + 16) * sizeof(int);
}

// position -> pair, and the pair's owning CTA
__device__ __forceinline__ int jd_pair(int x, int np, int P) { return x < P ? x : np - 1 - x; }
__device__ __forceinline__ int jd_prev(int x, int np) { return x == 0 ? 0 : (x == 1 ? np - 1 : x - 1); }
__device__ __forceinline__ int jd_next(int x, int np) { return x == 0 ? 0 : (x == np - 1 ? 1 : x + 1); }

__global__ void __launch_bounds__(kDsmThreads, 1) k_jacobi_dsm(JdsmArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char dsm[];
  const int n = a.n, np = a.np, P = a.P, PP = a.PP;
  const int me = (int)cluster.block_rank();
  const int k0 = me * PP;
  const int ns = max(0, min(PP, P - k0));  // own pairs
  const int nslot = 2 * ns;
  const int nbuf = 2 * PP + 2;
  const int ibuf0 = nbuf - 2;  // inbox buffers ibuf0 (positions < P), ibuf0 + 1 (>= P)
  float2* colA = (float2*)dsm;
  float2* colQ = colA + (size_t)nbuf * n;
  float2* alls = colQ + (size_t)nbuf * n;
  float2* rs = alls + P;
  float* allc = (float*)(rs + PP);
  float* rc = allc + P;
  float* red = rc + PP;  // [0] off, [1] dmax (published), [2..66) warp partials
  int* allp = (int*)(red + 66);
  int* allq = allp + P;
  int* rp = allq + P;
  int* rq = rp + PP;
  int* rbp = rq + PP;
  int* rbq = rbp + PP;
  int* tab = rbq + PP;        // 4 arrays of 2 PP: player/buffer x current/next
  int* misc = tab + 8 * PP;   // [0..1] inbox players, [2..15] schedule
  int* player = tab;
  int* bufof = tab + 2 * PP;
  int* nplayer = tab + 4 * PP;
  int* nbufof = tab + 6 * PP;

  // Fixed per CTA: own slot s stands at position pos(s); the slots whose
  // player leaves this CTA each round, and the slots that receive from an
  // inbox.  At most two of each (one per side).
  auto pos_of = [&](int s) { const int k = k0 + (s >> 1); return (s & 1) ? np - 1 - k : k; };
  auto slot_of = [&](int x) { const int k = jd_pair(x, np, P); return 2 * (k - k0) + (x >= P ? 1 : 0); };
  int n_out = 0, out_slot[2] = {-1, -1}, out_cta[2] = {0, 0}, out_box[2] = {0, 0};
  int n_in = 0, in_slot[2] = {-1, -1}, in_box[2] = {0, 0};
  for (int s = 0; s < nslot; ++s) {
    const int x = pos_of(s);
    const int d = jd_next(x, np);
    const int od = jd_pair(d, np, P) / PP;
    if (od != me && n_out < 2) {
      out_slot[n_out] = s;
      out_cta[n_out] = od;
      out_box[n_out] = d < P ? 0 : 1;
      ++n_out;
    }
    const int src = jd_prev(x, np);
    if (jd_pair(src, np, P) / PP != me && n_in < 2) {
      in_slot[n_in] = s;
      in_box[n_in] = x < P ? 0 : 1;
      ++n_in;
    }
  }

  // ---- load: position x starts with player x; Q starts as the identity
  for (int s = threadIdx.x; s < nslot; s += blockDim.x) {
    player[s] = pos_of(s);
    bufof[s] = s;
  }
  for (int t = threadIdx.x; t < nslot * n; t += blockDim.x) {
    const int s = t / n, i = t - s * n;
    const int pl = pos_of(s);
    if (pl < n) {
      const double2 v = a.A[(size_t)pl * a.lda + i];
      colA[(size_t)s * n + i] = make_float2((float)v.x, (float)v.y);
      colQ[(size_t)s * n + i] = make_float2(i == pl ? 1.f : 0.f, 0.f);
    }
  }
  __syncthreads();

  int sweep = 0;
  bool done = false;
  while (!done && sweep < a.max_sweeps) {
    for (int r = 0; r < np - 1; ++r) {
      // (a) rotations of the own pairs, published in rp/rq/rc/rs
      for (int j = threadIdx.x; j < ns; j += blockDim.x) {
        int p = player[2 * j], q = player[2 * j + 1];
        int bp = bufof[2 * j], bq = bufof[2 * j + 1];
        if (p > q) {
          int t = p; p = q; q = t;
          t = bp; bp = bq; bq = t;
        }
        float c = 1.f;
        float2 sv = make_float2(0.f, 0.f);
        if (q < n)
          jacobi_rotation<float>(colA[(size_t)bq * n + p], colA[(size_t)bp * n + p].x,
                                 colA[(size_t)bq * n + q].x, c, sv);
        rp[j] = p;
        rq[j] = q;
        rc[j] = c;
        rs[j] = sv;
        rbp[j] = bp;
        rbq[j] = bq;
      }
      cluster.sync();
      // (b) every rotation of the round, from the CTAs that own them
      for (int t = threadIdx.x; t < P; t += blockDim.x) {
        const int o = t / PP, jj = t - o * PP;
        allp[t] = cluster.map_shared_rank(rp, o)[jj];
        allq[t] = cluster.map_shared_rank(rq, o)[jj];
        allc[t] = cluster.map_shared_rank(rc, o)[jj];
        alls[t] = cluster.map_shared_rank(rs, o)[jj];
      }
      __syncthreads();
      // (c) A <- J^H A J on the own columns, Q <- Q J on the own Q columns
      const int nA = ns * P, nQ = ns * n;
      for (int t = threadIdx.x; t < nA + nQ; t += blockDim.x) {
        if (t < nA) {
          const int j = t / P, kk = t - j * P;
          const int pk = allp[kk], qk = allq[kk];
          if (pk >= n) continue;
          const int pl = rp[j], ql = rq[j];
          if (pl >= n) continue;
          const bool vk = qk < n, vl = ql < n;
          float2* cp = colA + (size_t)rbp[j] * n;
          float2* cq = colA + (size_t)rbq[j] * n;
          const float2 z = make_float2(0.f, 0.f);
          const float2 a00 = cp[pk];
          const float2 a01 = vl ? cq[pk] : z;
          const float2 a10 = vk ? cp[qk] : z;
          const float2 a11 = (vk && vl) ? cq[qk] : z;
          float2 y00, y01, y10, y11;
          jacobi_block<float>(a00, a01, a10, a11, allc[kk], alls[kk], rc[j], rs[j], y00, y01, y10,
                              y11);
          if (kk == k0 + j) {
            // rotated 2 x 2 diagonal block: real diagonal, zeroed pair element
            cp[pk] = make_float2(y00.x, 0.f);
            if (vk) {
              cq[qk] = make_float2(y11.x, 0.f);
              cq[pk] = z;
              cp[qk] = z;
            }
          } else {
            cp[pk] = y00;
            if (vl) cq[pk] = y01;
            if (vk) cp[qk] = y10;
            if (vk && vl) cq[qk] = y11;
          }
        } else {
          const int e = t - nA;
          const int j = e / n, i = e - j * n;
          if (rq[j] >= n) continue;  // pair with the dummy index: identity
          const float cl = rc[j];
          const float2 sl = rs[j];
          float2* qp = colQ + (size_t)rbp[j] * n;
          float2* qq = colQ + (size_t)rbq[j] * n;
          const float2 q0 = qp[i], q1 = qq[i];
          qp[i] = add<float>(scl<float>(q0, cl), mul<float>(q1, make_float2(-sl.x, sl.y)));
          qq[i] = add<float>(mul<float>(q0, sl), scl<float>(q1, cl));
        }
      }
      __syncthreads();
      // (d) players leaving this CTA: their columns into the neighbours' inboxes
      for (int o = 0; o < n_out; ++o) {
        const int b = bufof[out_slot[o]];
        const size_t dst = (size_t)(ibuf0 + out_box[o]) * n;
        float2* rA = cluster.map_shared_rank(colA, out_cta[o]);
        float2* rQ = cluster.map_shared_rank(colQ, out_cta[o]);
        if (player[out_slot[o]] < n) {
          for (int i = threadIdx.x; i < n; i += blockDim.x) {
            rA[dst + i] = colA[(size_t)b * n + i];
            rQ[dst + i] = colQ[(size_t)b * n + i];
          }
        }
        if (threadIdx.x == 0) cluster.map_shared_rank(misc, out_cta[o])[out_box[o]] = player[out_slot[o]];
      }
      cluster.sync();
      // (e) step every player to its next position
      for (int s = threadIdx.x; s < nslot; s += blockDim.x) {
        const int x = pos_of(s);
        const int src = jd_prev(x, np);
        if (jd_pair(src, np, P) / PP == me) {
          const int ss = slot_of(src);
          nplayer[s] = player[ss];
          nbufof[s] = bufof[ss];
        }
      }
      if (threadIdx.x == 0) {
        // arrivals take the buffers of the departures (equal counts)
        for (int i = 0; i < n_in; ++i) {
          nplayer[in_slot[i]] = misc[in_box[i]];
          nbufof[in_slot[i]] = i < n_out ? bufof[out_slot[i]] : ibuf0 + in_box[i];
        }
      }
      __syncthreads();
      for (int i = 0; i < n_in; ++i) {
        const int b = nbufof[in_slot[i]];
        const size_t src = (size_t)(ibuf0 + in_box[i]) * n;
        if (b != ibuf0 + in_box[i] && nplayer[in_slot[i]] < n) {
          for (int e = threadIdx.x; e < n; e += blockDim.x) {
            colA[(size_t)b * n + e] = colA[src + e];
            colQ[(size_t)b * n + e] = colQ[src + e];
          }
        }
      }
      {
        int* t = player; player = nplayer; nplayer = t;
        t = bufof; bufof = nbufof; nbufof = t;
      }
      __syncthreads();
    }
    ++sweep;
    // convergence: max |A_ij| (i != j) against max |A_ii| over every column
    float off = 0.f, dm = 0.f;
    for (int t = threadIdx.x; t < nslot * n; t += blockDim.x) {
      const int s = t / n, i = t - s * n;
      const int pl = player[s];
      if (pl >= n) continue;
      const float2 v = colA[(size_t)bufof[s] * n + i];
      if (i == pl) dm = fmaxf(dm, fabsf(v.x));
      else off = fmaxf(off, sqrtf(v.x * v.x + v.y * v.y));
    }
    for (int o = 16; o > 0; o >>= 1) {
      off = fmaxf(off, __shfl_xor_sync(0xffffffffu, off, o));
      dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    }
    if ((threadIdx.x & 31) == 0) {
      red[2 + (threadIdx.x >> 5)] = off;
      red[34 + (threadIdx.x >> 5)] = dm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float o2 = 0.f, d2 = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        o2 = fmaxf(o2, red[2 + w]);
        d2 = fmaxf(d2, red[34 + w]);
      }
      red[0] = o2;
      red[1] = d2;
    }
    cluster.sync();
    float goff = 0.f, gdm = 0.f;
    for (int c = 0; c < (int)cluster.num_blocks(); ++c) {
      const float* rr = cluster.map_shared_rank(red, c);
      goff = fmaxf(goff, rr[0]);
      gdm = fmaxf(gdm, rr[1]);
    }
    done = goff <= a.tol * fmaxf(gdm, 1e-30f);
    cluster.sync();  // every CTA has read the published values
  }

  // ---- results: column j of Q and A_jj for every own index j
  for (int t = threadIdx.x; t < nslot * n; t += blockDim.x) {
    const int s = t / n, i = t - s * n;
    const int pl = player[s];
    if (pl >= n) continue;
    const float2 v = colQ[(size_t)bufof[s] * n + i];
    a.Q[(size_t)pl * a.ldq + i] = make_double2((double)v.x, (double)v.y);
    if (i == pl) a.diag[pl] = (double)colA[(size_t)bufof[s] * n + i].x;
  }
  if (me == 0 && threadIdx.x == 0) {
    a.info[0] = 0;
    a.info[1] = sweep;
  }
  cluster.sync();
}

bool jacobi32_cluster(System& s, const double2* A, int64_t lda, int n, double tol, int max_sweeps,
                      double2* Q, int64_t ldq, double* diag, int* info, cudaStream_t st) {
  (void)s;
  // PWH_JACOBI_GLOBAL=1 in the environment selects the global-memory kernel
  static const bool off = [] {
    const char* e = std::getenv("PWH_JACOBI_GLOBAL");
    return e && e[0] == '1';
  }();
  if (off || n < 4) return false;
  const int np = n + (n & 1), P = np / 2;
  const int PP = (P + kDsmCluster - 1) / kDsmCluster;
  const size_t smem = jdsm_smem_bytes(n, P, PP);
  if (smem > 220 * 1024) return false;
  static std::once_flag attr_once;
  static bool attr_ok = false;
  std::call_once(attr_once, [] {
    attr_ok = cudaFuncSetAttribute(k_jacobi_dsm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   227 * 1024) == cudaSuccess &&
              cudaFuncSetAttribute(k_jacobi_dsm, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                  cudaSuccess;
    cudaGetLastError();
  });
  if (!attr_ok) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kDsmCluster);
  cfg.blockDim = dim3(kDsmThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kDsmCluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // can one cluster of this size and shared memory be resident?  (cached per size)
  {
    static std::mutex mu;
    static size_t fits_upto = 0, fails_from = ~size_t(0);
    std::lock_guard<std::mutex> lock(mu);
    if (smem > fits_upto) {
      if (smem >= fails_from) return false;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)k_jacobi_dsm, &cfg) != cudaSuccess ||
          nclusters < 1) {
        cudaGetLastError();
        fails_from = smem;
        return false;
      }
      fits_upto = smem;
    }
  }
  JdsmArgs a;
  a.A = A; a.lda = lda; a.Q = Q; a.ldq = ldq; a.diag = diag; a.info = info;
  a.n = n; a.np = np; a.P = P; a.PP = PP; a.max_sweeps = max_sweeps; a.tol = (float)tol;
  PWH_CUDA(cudaLaunchKernelEx(&cfg, k_jacobi_dsm, a));
  note_launch();
  return true;
}

}  // namespace pwh
