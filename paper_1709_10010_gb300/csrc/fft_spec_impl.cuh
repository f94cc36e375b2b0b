// FFT passes specialised at compile time for cubic boxes of common sizes.
// Same data layout and twiddle table as the generic passes in fft.cu
// (k_zinv, k_plane, k_zfwd), but every 1D transform is a two-pass four-step
// FFT in natural order whose small DFTs run in registers with compile-time
// indices (no digit-reversed scatter, two shared-memory passes per
// transform instead of one per radix stage).
#pragma once
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "fft_device.cuh"
#include "fft_spec.cuh"

namespace pwh {

struct CPlan {
  int ns;
  int R[kMaxStages];
  int M[kMaxStages];
  int L[kMaxStages];
};

constexpr CPlan make_cplan(int n) {
  CPlan p{};
  int r = n, ns = 0;
  int rad[kMaxStages] = {};
  while (r % 4 == 0) { rad[ns++] = 4; r /= 4; }
  while (r % 2 == 0) { rad[ns++] = 2; r /= 2; }
  while (r % 3 == 0) { rad[ns++] = 3; r /= 3; }
  while (r % 5 == 0) { rad[ns++] = 5; r /= 5; }
  p.ns = ns;
  int m = 1;
  for (int s = 0; s < ns; ++s) {
    p.R[s] = rad[s];
    p.M[s] = m;
    m *= rad[s];
    p.L[s] = m;
  }
  return p;
}

// Stages S.. of nfft transforms of length N (unit element stride, transform f
// at data + f * fstride), all threads of the block; ends with __syncthreads().
template <typename T, bool INV, int N, int S>
__device__ __forceinline__ void fft_stages(cx<T>* data, int nfft, int fstride, const cx<T>* tw) {
  constexpr CPlan P = make_cplan(N);
  if constexpr (S < P.ns) {
    constexpr int s = INV ? S : P.ns - 1 - S;
    constexpr int R = P.R[s], M = P.M[s], L = P.L[s];
    constexpr int nbf = N / R, twstep = N / L;
    const T sg = INV ? (T)1 : (T)-1;
    const int total = nfft * nbf;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int f = t / nbf, j = t - f * nbf;
      const int g = j / M, k1 = j - g * M;
      butterfly<T, R, INV>(data + f * fstride + g * L + k1, 1, M, k1, twstep, tw, sg);
    }
    __syncthreads();
    fft_stages<T, INV, N, S + 1>(data, nfft, fstride, tw);
  }
}

// ---- natural-order transforms: N = N1 N2 in two passes (the four-step
// factorisation), each pass a batch of small DFTs held in registers.
//   pass 1: for each n2 < N2, the N1-point DFT over x[N2 n1 + n2], times
//           w_N^(n2 k1), back to x[N2 k1 + n2];
//   pass 2: for each k1 < N1, the N2-point DFT over x[N2 k1 + n2], to
//           x[k1 + N1 k2].
// The small DFTs are the same mixed-radix DIT (input in the digit-reversed
// order of make_cplan, a free renaming of registers) with every index a
// compile-time constant; twiddles come from the length-N table tw.
struct RevTab {
  int v[32];
};
// position q of the DIT input holds element v[q] (digits of q, recombined
// in reverse radix order)
constexpr RevTab make_rev(int n) {
  const CPlan p = make_cplan(n);
  RevTab t{};
  for (int q = 0; q < n; ++q) {
    int rem = q, dig[kMaxStages] = {};
    for (int s = 0; s < p.ns; ++s) {
      dig[s] = rem % p.R[s];
      rem /= p.R[s];
    }
    int acc = p.ns ? dig[0] : 0;
    for (int s = 1; s < p.ns; ++s) acc = dig[s] + p.R[s] * acc;
    t.v[q] = acc;
  }
  return t;
}
// a factor N1 of N near sqrt(N) with N1, N / N1 <= 16
constexpr int fft_factor(int n) {
  int best = 1;
  for (int d = 2; d <= 16; ++d)
    if (n % d == 0 && n / d <= 16 && (best == 1 || (d <= n / d && d > best))) best = d;
  return best;
}

template <typename T, int R, bool INV, int NT, int S>
__device__ __forceinline__ void reg_stages(cx<T>* a, const cx<T>* tw) {
  constexpr CPlan P = make_cplan(R);
  if constexpr (S < P.ns) {
    constexpr int Rs = P.R[S], M = P.M[S], L = P.L[S];
    constexpr int twstep = NT / L;
    const T sg = INV ? (T)1 : (T)-1;
#pragma unroll
    for (int g = 0; g < R / L; ++g)
#pragma unroll
      for (int k1 = 0; k1 < M; ++k1) {
        cx<T> b[Rs];
#pragma unroll
        for (int q = 0; q < Rs; ++q) b[q] = a[g * L + k1 + q * M];
        if (k1 != 0) {
#pragma unroll
          for (int q = 1; q < Rs; ++q) {
            cx<T> w = tw[q * k1 * twstep];
            w.y *= sg;
            b[q] = mul<T>(b[q], w);
          }
        }
        dft<T, Rs>(b, sg);
#pragma unroll
        for (int q = 0; q < Rs; ++q) a[g * L + k1 + q * M] = b[q];
      }
    reg_stages<T, R, INV, NT, S + 1>(a, tw);
  }
}
// In-register DFT of length R (natural order in and out) with sign +1 (INV)
// or -1; tw[t] = exp(2 pi i t / NT), R | NT.
template <typename T, int R, bool INV, int NT>
__device__ __forceinline__ void dft_reg(cx<T>* x, const cx<T>* tw) {
  constexpr RevTab rv = make_rev(R);
  cx<T> a[R];
#pragma unroll
  for (int q = 0; q < R; ++q) a[q] = x[rv.v[q]];
  reg_stages<T, R, INV, NT, 0>(a, tw);
#pragma unroll
  for (int k = 0; k < R; ++k) x[k] = a[k];
}

// nfft transforms of length N in shared memory (transform f at data + f
// fstride, unit stride), natural order in and out; all threads of the block;
// ends with __syncthreads().
template <typename T, bool INV, int N>
__device__ __forceinline__ void fft_nat(cx<T>* data, int nfft, int fstride, const cx<T>* tw) {
  constexpr int N1 = fft_factor(N), N2 = N / N1;
  static_assert(N1 > 1 && N1 <= 16 && N2 <= 16, "factor");
  const T sg = INV ? (T)1 : (T)-1;
  for (int t = threadIdx.x; t < nfft * N2; t += blockDim.x) {
    const int f = t / N2, n2 = t - f * N2;
    cx<T>* xf = data + f * fstride;
    cx<T> v[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) v[n1] = xf[N2 * n1 + n2];
    dft_reg<T, N1, INV, N>(v, tw);
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) {
      cx<T> w = tw[n2 * k1];
      w.y *= sg;
      v[k1] = mul<T>(v[k1], w);
    }
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) xf[N2 * k1 + n2] = v[k1];
  }
  __syncthreads();
  // pass 2 writes other positions than it reads: whole transforms per round,
  // loads and stores separated by a barrier
  const int per = blockDim.x / N1;
  const int fl = threadIdx.x / N1, k1 = threadIdx.x - fl * N1;
  for (int f0 = 0; f0 < nfft; f0 += per) {
    const int f = f0 + fl;
    const bool act = fl < per && f < nfft;
    cx<T> w[N2];
    if (act) {
      const cx<T>* xf = data + f * fstride + N2 * k1;
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) w[n2] = xf[n2];
      dft_reg<T, N2, INV, N>(w, tw);
    }
    __syncthreads();
    if (act) {
      cx<T>* xf = data + f * fstride + k1;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) xf[N1 * k2] = w[k2];
    }
  }
  __syncthreads();
}

template <typename T, int N>
__global__ void __launch_bounds__(256) ks_zinv(const double2* __restrict__ psi, int64_t ldp,
                                               const int32_t* __restrict__ stick_off,
                                               const int32_t* __restrict__ stick_of,
                                               const int16_t* __restrict__ zpos, int nsticks,
                                               int tw_off, int perm_off,
                                               const cx<T>* __restrict__ tw_g,
                                               const int16_t* __restrict__ perm_g,
                                               cx<T>* __restrict__ W, int64_t wband, int spb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int ld = N + 1;
  cx<T>* buf = (cx<T>*)smem_raw;
  cx<T>* tw = buf + spb * ld;
  int16_t* irev = (int16_t*)(tw + N);
  const int b = blockIdx.y;
  const int s0 = blockIdx.x * spb;
  const int ns = min(spb, nsticks - s0);
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    tw[t] = tw_g[tw_off + t];
    irev[t] = perm_g[perm_off + t];
  }
  for (int t = threadIdx.x; t < spb * ld; t += blockDim.x) buf[t] = mk<T>(0, 0);
  __syncthreads();
  const int i0 = stick_off[s0], i1 = stick_off[s0 + ns];
  const double2* src = psi + (size_t)b * ldp;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x)
    buf[(stick_of[i] - s0) * ld + zpos[i]] = widen_from64<T>(src[i]);
  __syncthreads();
  fft_nat<T, true, N>(buf, ns, ld, tw);
  cx<T>* dst = W + (size_t)b * wband;
  for (int t = threadIdx.x; t < N * spb; t += blockDim.x) {
    const int z = t / spb, s = t - z * spb;
    if (s < ns) dst[(size_t)z * nsticks + s0 + s] = buf[s * ld + z];
  }
}

// ---- the plane pass: per (z-plane, band) the y transforms on the columns
// that hold sticks, the x transforms on every row with V(r) applied between
// them, each 1D transform the four-step N = N1 N2 of fft_nat written out as
// two register passes whose loads and stores do the data movement too:
//   y inverse  pass 1 loads the plane's sticks from W through stick_at (zero
//              where no stick), pass 2 in place in C[column][y];
//   x inverse  pass 1 loads the columns of C through xcol (zero elsewhere),
//              pass 2 in registers, times V(r), straight into
//   x forward  pass 1 of the transposed factorisation N = N2 N1 (the
//              registers of a thread already hold its inputs), then pass 2
//              stores only the columns back into C;
//   y forward  pass 1 in place, pass 2 stores only the sticks back into W.
// No zero fill, scatter or gather pass of its own; row chunks of `rows` rows
// bound the shared memory.

// Four-step pass 1 on registers: v[n1] = x[N2 n1 + n2] -> w^(n2 k1) DFT_N1(v)[k1]
// (w = e^{+-2 pi i/N}), natural order out.  tw4[k1 N2 + n2] = e^{2 pi i n2 k1/N}:
// threads with consecutive n2 read consecutive entries (no bank conflicts).
template <typename T, int N, bool INV>
__device__ __forceinline__ void fs_pass1(cx<T>* v, int n2, const cx<T>* tw, const cx<T>* tw4) {
  constexpr int N1 = fft_factor(N), N2 = N / N1;
  const T sg = INV ? (T)1 : (T)-1;
  dft_reg<T, N1, INV, N>(v, tw);
#pragma unroll
  for (int k1 = 1; k1 < N1; ++k1) {
    cx<T> w = tw4[k1 * N2 + n2];
    w.y *= sg;
    v[k1] = mul<T>(v[k1], w);
  }
}

// Four-step pass 2 in place on nf transforms of shared memory (transform f at
// data + f ld): x[N2 k1 + n2] -> x[k1 + N1 k2], rounds of whole transforms,
// each round loads, synchronises, then stores; `post(f, x, value)` maps an
// output before it is stored.  FFAST: neighbouring threads take neighbouring
// transforms (odd ld: conflict-free shared-memory access), else neighbouring
// k1 (neighbouring x, for coalesced global reads in post).  Ends with
// __syncthreads().
template <typename T, int N, int NT, bool INV, bool FFAST, class Post>
__device__ __forceinline__ void fs_pass2_inplace(cx<T>* data, int nf, int ld, const cx<T>* tw,
                                                 Post post) {
  constexpr int N1 = fft_factor(N), N2 = N / N1;
  constexpr int per = NT / N1;
  const int fl = FFAST ? (int)threadIdx.x % per : (int)threadIdx.x / N1;
  const int k1 = FFAST ? (int)threadIdx.x / per : (int)threadIdx.x - fl * N1;
  for (int f0 = 0; f0 < nf; f0 += per) {
    const int f = f0 + fl;
    const bool act = fl < per && k1 < N1 && f < nf;
    cx<T> w[N2];
    if (act) {
      const cx<T>* xf = data + f * ld + N2 * k1;
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) w[n2] = xf[n2];
      dft_reg<T, N2, INV, N>(w, tw);
    }
    __syncthreads();
    if (act) {
      cx<T>* xf = data + f * ld + k1;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) xf[N1 * k2] = post(f, k1 + N1 * k2, w[k2]);
    }
  }
  __syncthreads();
}

// The middle of the row transforms, in place on nf rows of shared memory (row
// f at data + f ld): pass 2 of the inverse transform, times V(r), then pass 1
// of the forward transform in the transposed factorisation N = N2 N1.  Thread
// (row, k1) loads x[N2 k1 + n2] (n2 < N2) and after the inverse DFT over n2
// holds the natural-order values x[k1 + N1 m] (m < N2), which are exactly the
// inputs of the forward transform's first pass for residue k1 mod N1: the
// forward N2-point DFT over m and the twiddle w^(k1 j) give Y[k1][j], stored
// at k1 + N1 j.  Ends with __syncthreads().
template <typename T, int N, int NT>
__device__ __forceinline__ void fs_rows_mid(cx<T>* data, int nf, int ld, const cx<T>* tw,
                                            const cx<T>* tw4, const T* Vy) {
  constexpr int N1 = fft_factor(N), N2 = N / N1;
  constexpr int per = NT / N1;
  const int fl = (int)threadIdx.x / N1;
  const int k1 = (int)threadIdx.x - fl * N1;
  for (int f0 = 0; f0 < nf; f0 += per) {
    const int f = f0 + fl;
    const bool act = fl < per && f < nf;
    cx<T> w[N2];
    if (act) {
      const cx<T>* xf = data + f * ld + N2 * k1;
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) w[n2] = xf[n2];
      dft_reg<T, N2, true, N>(w, tw);
      const T* vr = Vy + (size_t)f * N + k1;
#pragma unroll
      for (int m = 0; m < N2; ++m) w[m] = scl<T>(w[m], vr[N1 * m]);
      dft_reg<T, N2, false, N>(w, tw);
#pragma unroll
      for (int j = 1; j < N2; ++j) {
        cx<T> t = tw4[k1 * N2 + j];
        t.y = -t.y;
        w[j] = mul<T>(w[j], t);
      }
    }
    __syncthreads();
    if (act) {
      cx<T>* xf = data + f * ld + k1;
#pragma unroll
      for (int j = 0; j < N2; ++j) xf[N1 * j] = w[j];
    }
  }
  __syncthreads();
}

template <typename T, int N, int NT>
__global__ void __launch_bounds__(NT) ks_plane(cx<T>* __restrict__ W, int64_t wband, int nsticks,
                                               int ncols, const int32_t* __restrict__ stick_at,
                                               const int16_t* __restrict__ xcol_g,
                                               const T* __restrict__ V, int tw_off,
                                               const cx<T>* __restrict__ tw_g, int rows) {
  constexpr int N1 = fft_factor(N), N2 = N / N1, LD = N + 1;
  static_assert(N1 > 1 && N1 <= 16 && N2 <= 16, "factor");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* C = (cx<T>*)smem_raw;             // ncols x LD: columns along y
  cx<T>* R = C + (size_t)ncols * LD;       // rows x LD: rows along x
  cx<T>* tw = R + (size_t)rows * LD;       // e^{2 pi i t/N}
  cx<T>* tw4 = tw + N;                     // [k1][n2]: e^{2 pi i n2 k1/N}
  int16_t* xcol = (int16_t*)(tw4 + N);     // column of each x, -1 if none
  const int z = blockIdx.x, b = blockIdx.y;
  cx<T>* plane = W + (size_t)b * wband + (size_t)z * nsticks;
  for (int t = threadIdx.x; t < N; t += NT) {
    tw[t] = tw_g[tw_off + t];
    tw4[t] = tw_g[tw_off + (t % N2) * (t / N2)];
    xcol[t] = xcol_g[t];
  }
  __syncthreads();
  const cx<T> zero = mk<T>(0, 0);

  // ---- y inverse: sticks -> C
  for (int t = threadIdx.x; t < ncols * N2; t += NT) {
    const int c = t / N2, n2 = t - c * N2;
    const int32_t* sa = stick_at + (size_t)c * N + n2;
    cx<T> v[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const int st = sa[N2 * n1];
      v[n1] = st >= 0 ? plane[st] : zero;
    }
    fs_pass1<T, N, true>(v, n2, tw, tw4);
    cx<T>* cc = C + c * LD + n2;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) cc[N2 * k1] = v[k1];
  }
  __syncthreads();
  fs_pass2_inplace<T, N, NT, true, true>(C, ncols, LD, tw, [](int, int, cx<T> v) { return v; });

  // ---- rows: x inverse, times V, x forward; keep the columns
  const T* Vz = V + (size_t)z * N * N;
  for (int y0 = 0; y0 < N; y0 += rows) {
    const int nr = min(rows, N - y0);
    for (int t = threadIdx.x; t < nr * N2; t += NT) {
      const int r = t / N2, n2 = t - r * N2;
      cx<T> v[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) {
        const int c = xcol[N2 * n1 + n2];
        v[n1] = c >= 0 ? C[c * LD + y0 + r] : zero;
      }
      fs_pass1<T, N, true>(v, n2, tw, tw4);
      cx<T>* rr = R + r * LD + n2;
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) rr[N2 * k1] = v[k1];
    }
    __syncthreads();
    fs_rows_mid<T, N, NT>(R, nr, LD, tw, tw4, Vz + (size_t)y0 * N);
    // forward pass 2 (N1-point DFTs over k1): X[j + N2 l], only the columns
    for (int t = threadIdx.x; t < nr * N2; t += NT) {
      const int r = t % nr, j = t / nr;  // neighbouring rows: conflict-free
      const cx<T>* rr = R + r * LD + N1 * j;
      cx<T> v[N1];
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) v[k1] = rr[k1];
      dft_reg<T, N1, false, N>(v, tw);
#pragma unroll
      for (int l = 0; l < N1; ++l) {
        const int c = xcol[j + N2 * l];
        if (c >= 0) C[c * LD + y0 + r] = v[l];
      }
    }
    __syncthreads();
  }

  // ---- y forward: C -> sticks
  for (int t = threadIdx.x; t < ncols * N2; t += NT) {
    const int c = t / N2, n2 = t - c * N2;
    cx<T>* cc = C + c * LD + n2;
    cx<T> v[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) v[n1] = cc[N2 * n1];
    fs_pass1<T, N, false>(v, n2, tw, tw4);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) cc[N2 * k1] = v[k1];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ncols * N1; t += NT) {
    const int c = t / N1, k1 = t - c * N1;
    const cx<T>* cc = C + c * LD + N2 * k1;
    cx<T> w[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) w[n2] = cc[n2];
    dft_reg<T, N2, false, N>(w, tw);
    const int32_t* sa = stick_at + (size_t)c * N + k1;
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const int st = sa[N1 * k2];
      if (st >= 0) plane[st] = w[k2];
    }
  }
}

// Shared memory of the plane pass for `rows` rows per chunk.
template <typename T, int N> constexpr size_t ks_plane_smem(int ncols, int rows) {
  return ((size_t)(ncols + rows) * (N + 1) + 2 * N) * sizeof(cx<T>) + N * sizeof(int16_t);
}

template <typename T, int N>
__global__ void __launch_bounds__(256) ks_zfwd(const cx<T>* __restrict__ W, int64_t wband,
                                               const int32_t* __restrict__ stick_off,
                                               const int32_t* __restrict__ stick_of,
                                               const int16_t* __restrict__ zpos, int nsticks,
                                               int tw_off, int perm_off,
                                               const cx<T>* __restrict__ tw_g,
                                               const int16_t* __restrict__ perm_g,
                                               const double* __restrict__ kin,
                                               const double2* __restrict__ psi, int64_t ldp,
                                               double2* __restrict__ hpsi, int64_t ldh, int spb,
                                               const float2* __restrict__ vnl, int64_t ldv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int ld = N + 1;
  cx<T>* buf = (cx<T>*)smem_raw;
  cx<T>* tw = buf + spb * ld;
  int16_t* irev = (int16_t*)(tw + N);
  const int b = blockIdx.y;
  const int s0 = blockIdx.x * spb;
  const int ns = min(spb, nsticks - s0);
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    tw[t] = tw_g[tw_off + t];
    irev[t] = perm_g[perm_off + t];
  }
  const cx<T>* src = W + (size_t)b * wband;
  for (int t = threadIdx.x; t < N * spb; t += blockDim.x) {
    const int z = t / spb, s = t - z * spb;
    if (s < ns) buf[s * ld + z] = src[(size_t)z * nsticks + s0 + s];
  }
  __syncthreads();
  fft_nat<T, false, N>(buf, ns, ld, tw);
  const int i0 = stick_off[s0], i1 = stick_off[s0 + ns];
  const double2* pb = psi + (size_t)b * ldp;
  double2* hb = hpsi + (size_t)b * ldh;
  const float2* vb = vnl ? vnl + (size_t)b * ldv : nullptr;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const cx<T> v = buf[(stick_of[i] - s0) * ld + zpos[i]];
    const double2 p = pb[i];
    const double k = kin[i];
    double2 h = kin_plus<T>(k, p, v);
    if (vb) {
      const float2 u = vb[i];
      h.x += (double)u.x;
      h.y += (double)u.y;
    }
    hb[i] = h;
  }
}

// Rows per chunk of the plane pass, autotuned: the candidates are equal
// chunkings of the N rows whose shared memory fits (one to six chunks); on the
// first use per (N, precision, column count) with a batch of at least 8 bands,
// each is timed with CUDA events (two launches, the second timed) on a scratch
// copy of the batch's stick buffer, and the fastest is kept for the rest of
// the process.  Before that, and while the stream is being captured, the size
// heuristic decides: the fewest chunks that keep two blocks per SM, else one.
template <typename T, int N> int plane_rows_heuristic(int ncols) {
  int rows = N;
  for (size_t cap : {(size_t)110 * 1024, (size_t)220 * 1024}) {
    int r = N;
    while (r > 1 && ks_plane_smem<T, N>(ncols, r) > cap) --r;
    const int chunks = (N + r - 1) / r;
    rows = (N + chunks - 1) / chunks;
    if (ks_plane_smem<T, N>(ncols, rows) <= cap && (rows >= 32 || rows == N)) break;
  }
  if (ks_plane_smem<T, N>(ncols, rows) > 227 * 1024)
    throw Error{PWH_ERR_ARG, "FFT plane does not fit in shared memory"};
  return rows;
}

template <typename T, int N> int plane_rows(System& s, const PassArgs& a) {
  static std::mutex mu;
  static std::map<int, int> chosen;  // ncols -> rows
  std::lock_guard<std::mutex> lock(mu);
  auto it = chosen.find(s.ncols);
  if (it != chosen.end()) return it->second;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  PWH_CUDA(cudaStreamIsCapturing(a.st, &cap));
  const int heur = plane_rows_heuristic<T, N>(s.ncols);
  // a capture cannot time; a batch of a few bands would time launch overhead
  if (cap != cudaStreamCaptureStatusNone || a.bb < 8) return heur;
  std::vector<int> cands;
  for (int c = 1; c <= 6; ++c) {
    const int r = (N + c - 1) / c;
    if (ks_plane_smem<T, N>(s.ncols, r) <= 227 * 1024 &&
        (cands.empty() || cands.back() != r))
      cands.push_back(r);
  }
  int best = heur;
  if (cands.size() > 1) {
    const size_t bytes = (size_t)a.bb * a.wband * sizeof(cx<T>);
    ensure(s.ws_tune, bytes);
    cx<T>* Wt = (cx<T>*)s.ws_tune.p;
    PWH_CUDA(cudaMemcpyAsync(Wt, a.W, bytes, cudaMemcpyDeviceToDevice, a.st));
    cudaEvent_t e0, e1;
    PWH_CUDA(cudaEventCreate(&e0));
    PWH_CUDA(cudaEventCreate(&e1));
    float best_ms = 0.f;
    for (int r : cands) {
      const size_t smem = ks_plane_smem<T, N>(s.ncols, r);
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        if (rep == 1) PWH_CUDA(cudaEventRecord(e0, a.st));
        ks_plane<T, N, 512><<<dim3(N, a.bb), 512, smem, a.st>>>(
            Wt, a.wband, s.nsticks, s.ncols, s.d_stick_at, s.d_xcol, (const T*)a.V,
            s.plan[0].tw_off, (const cx<T>*)a.tw, r);
        PWH_LAUNCH_CHECK();
      }
      PWH_CUDA(cudaEventRecord(e1, a.st));
      PWH_CUDA(cudaEventSynchronize(e1));
      PWH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (best_ms == 0.f || ms < best_ms) {
        best_ms = ms;
        best = r;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  chosen[s.ncols] = best;
  return best;
}

template <typename T, int N> void spec_launch(SpecPass pass, System& s, const PassArgs& a) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(ks_zinv<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(ks_plane<T, N, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(ks_zfwd<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  const cx<T>* tw = (const cx<T>*)a.tw;
  cx<T>* W = (cx<T>*)a.W;
  const dim3 gz((s.nsticks + a.spb - 1) / a.spb, a.bb);
  switch (pass) {
    case SPEC_ZINV:
      ks_zinv<T, N><<<gz, 256, a.zsmem, a.st>>>(a.psi, a.ldp, s.d_stick_off, s.d_stick_of, s.d_zpos,
                                                 s.nsticks, s.plan[2].tw_off, s.plan[2].perm_off, tw,
                                                 s.d_perm, W, a.wband, a.spb);
      break;
    case SPEC_PLANE: {
      const int rows = plane_rows<T, N>(s, a);
      ks_plane<T, N, 512><<<dim3(N, a.bb), 512, ks_plane_smem<T, N>(s.ncols, rows), a.st>>>(
          W, a.wband, s.nsticks, s.ncols, s.d_stick_at, s.d_xcol, (const T*)a.V, s.plan[0].tw_off,
          tw, rows);
      break;
    }
    case SPEC_ZFWD:
      ks_zfwd<T, N><<<gz, 256, a.zsmem, a.st>>>(W, a.wband, s.d_stick_off, s.d_stick_of, s.d_zpos,
                                                 s.nsticks, s.plan[2].tw_off, s.plan[2].perm_off, tw,
                                                 s.d_perm, s.d_kin, a.psi, a.ldp, a.hpsi, a.ldh, a.spb,
                                                 a.vnl, a.ldv);
      break;
  }
  PWH_LAUNCH_CHECK();
}

template <typename T> bool spec_pass(SpecPass pass, System& s, const PassArgs& a) {
  if (s.n1 != s.n2 || s.n2 != s.n3) return false;
  switch (s.n1) {
#define PWH_SPEC_CASE(n) \
  case n: spec_launch<T, n>(pass, s, a); return true;
    PWH_SPEC_SIZES(PWH_SPEC_CASE)
#undef PWH_SPEC_CASE
    default: return false;
  }
}

}  // namespace pwh
