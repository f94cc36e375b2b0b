// Shared internals of libpwh: status plumbing, complex helpers, the system
// object.  Host and device code.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pwh.h"

namespace pwh {

// ---------------------------------------------------------------- errors ----
void set_error(const std::string& msg);

struct Error {
  pwh_status st;
  std::string msg;
};

#define PWH_CHECK_ARG(cond, msg)                                   \
  do {                                                             \
    if (!(cond)) throw ::pwh::Error{PWH_ERR_ARG, std::string(msg)}; \
  } while (0)

#define PWH_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      throw ::pwh::Error{e_ == cudaErrorMemoryAllocation ? PWH_ERR_OOM : PWH_ERR_CUDA,  \
                         std::string(#call) + ": " + cudaGetErrorString(e_)};           \
    }                                                                                   \
  } while (0)

// Every kernel launch site ends with PWH_LAUNCH_CHECK(): it checks the launch
// and counts it (pwh_launch_count).
void note_launch();
void note_launches(long long n);  // kernels launched through a replayed CUDA graph
long long launch_counter();       // launches made by the calling thread
#define PWH_LAUNCH_CHECK()          \
  do {                              \
    ::pwh::note_launch();           \
    PWH_CUDA(cudaGetLastError());   \
  } while (0)

// ------------------------------------------------------------- complex ------
template <typename T> struct cplx;
template <> struct cplx<double> { using t = double2; };
template <> struct cplx<float> { using t = float2; };
template <typename T> using cx = typename cplx<T>::t;

template <typename T> __host__ __device__ __forceinline__ cx<T> mk(T r, T i) {
  cx<T> z; z.x = r; z.y = i; return z;
}
template <typename T> __host__ __device__ __forceinline__ cx<T> add(cx<T> a, cx<T> b) {
  return mk<T>(a.x + b.x, a.y + b.y);
}
template <typename T> __host__ __device__ __forceinline__ cx<T> sub(cx<T> a, cx<T> b) {
  return mk<T>(a.x - b.x, a.y - b.y);
}
template <typename T> __host__ __device__ __forceinline__ cx<T> mul(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __host__ __device__ __forceinline__ cx<T> mulc(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T> __host__ __device__ __forceinline__ cx<T> scl(cx<T> a, T s) {
  return mk<T>(a.x * s, a.y * s);
}

// --------------------------------------------------- format conversion ----
// IEEE 754 binary64 <-> binary32 conversions with integer operations only: on
// this GPU conversions to and from FP64 issue on the narrow FP64 pipe, which
// made them the bottleneck of kernels that widen or narrow every element.
// d2f_rn rounds to nearest, ties to even (subnormal results included, overflow
// to infinity, NaN stays NaN); f2d is exact.
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = b & 0xfffffffffffffull;
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m ? 0x400000u : 0u));
  const int ef = e - 1023 + 127;
  if (ef > 0) {
    if (ef >= 255) return __uint_as_float(sign | 0x7f800000u);
    // 23 kept fraction bits, 29 dropped; a carry out of the fraction moves
    // into the exponent (up to infinity), as the encoding intends
    unsigned q = (unsigned)(m >> 29);
    const unsigned rem = (unsigned)(m & 0x1fffffffu);
    q += (rem > 0x10000000u || (rem == 0x10000000u && (q & 1u))) ? 1u : 0u;
    return __uint_as_float(sign | (((unsigned)ef << 23) + q));
  }
  // binary32 subnormal or zero: value = M 2^(e - 1075), unit 2^-149
  if (e == 0) return __uint_as_float(sign);
  const unsigned long long M = m | (1ull << 52);
  const int sh = 926 - e;  // >= 30
  if (sh >= 64) return __uint_as_float(sign);
  unsigned long long q = M >> sh;
  const unsigned long long rem = M & ((1ull << sh) - 1), half = 1ull << (sh - 1);
  q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
  return __uint_as_float(sign | (unsigned)q);
}
__device__ __forceinline__ double f2d(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  int e = (int)((b >> 23) & 0xff);
  unsigned m = b & 0x7fffffu;
  if (e == 255)
    return __longlong_as_double((long long)(sign | (0x7ffull << 52) | ((unsigned long long)m << 29)));
  if (e == 0) {
    if (m == 0) return __longlong_as_double((long long)sign);
    const int sh = __clz(m) - 8;  // normalise the subnormal fraction
    m = (m << sh) & 0x7fffffu;
    e = 1 - sh;
  }
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)(e - 127 + 1023) << 52) | ((unsigned long long)m << 29)));
}
__device__ __forceinline__ float2 d2f_rn(double2 z) { return make_float2(d2f_rn(z.x), d2f_rn(z.y)); }
__device__ __forceinline__ double2 f2d(float2 z) { return make_double2(f2d(z.x), f2d(z.y)); }

// ------------------------------------------------------------- FFT plan -----
constexpr int kMaxStages = 10;
constexpr int kMaxFft = 512;

// One 1D transform length N = prod(radix).  Stage s combines sub-transforms of
// length M[s] into length L[s] = M[s] * radix[s] (decimation in time); the
// decimation-in-frequency transform runs the stages in reverse.
struct FftPlan {
  int n;
  int nstages;
  int radix[kMaxStages];
  int M[kMaxStages];
  int L[kMaxStages];
  int tw_off;    // offset of this length's table e^{+2 pi i t/n}, t in [0,n)
  int perm_off;  // offset of its digit-reversal table rev[p]
};

// ------------------------------------------------------------- system -------
template <typename T> struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
};

struct DavWs;
void free_davidson_ws(DavWs* w);

// Optional per-family kernel timing with CUDA events on the system's stream.
enum KernelFamily {
  KF_FFT_ZINV64 = 0, KF_FFT_PLANE64, KF_FFT_ZFWD64, KF_FFT_ZINV32, KF_FFT_PLANE32, KF_FFT_ZFWD32,
  KF_TC_BECP, KF_TC_BACK, KF_GEMM_FP64, KF_GEMM_FP32, KF_JACOBI, KF_CHOLQR, KF_JACOBI32,
  KF_GEMM_OZ, KF_GEMM_X3, KF_COUNT
};
extern const char* const kKernelFamilyName[KF_COUNT];

struct KernelTimer {
  bool on = false;
  int depth = 0;  // nested scopes are attributed to the outermost family
  double ms[KF_COUNT] = {};
  long long n[KF_COUNT] = {};
  double flops[KF_COUNT] = {};  // algorithmic work of the timed launches
  double bytes[KF_COUNT] = {};
  struct Pending { int fam; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get();
  void resolve();  // waits for the recorded events, accumulates, recycles
  void reset();
  ~KernelTimer();
};

struct System {
  // description
  double lattice[9];
  double kpoint[3];
  double ecut;
  int n1, n2, n3;
  int precision;
  cudaStream_t stream;

  // basis (host)
  int64_t npw = 0;
  std::vector<int32_t> miller;   // public order, npw*3
  std::vector<double> kin_pub;   // public order
  std::vector<int32_t> int_to_pub;
  int nsticks = 0, ncols = 0;
  std::vector<int32_t> stick_off;  // nsticks+1, internal offsets
  std::vector<int32_t> stick_col, stick_y;  // column index, y grid index
  std::vector<int32_t> col_x;      // x grid index of each column
  int nshell = 0;                  // shells of equal |k+G|^2 (public-order rule)
  std::vector<int32_t> shell_pub;  // shell of each public plane wave
  std::vector<double> Tshell_h;    // 1/2|k+G|^2 of each shell

  // device: maps and tables
  int32_t* d_int_to_pub = nullptr;
  double* d_kin = nullptr;          // internal order
  int32_t* d_stick_off = nullptr;
  int32_t* d_stick_of = nullptr;    // stick of each internal plane wave
  int16_t* d_zpos = nullptr;        // m3 mod N3 of each internal plane wave
  int32_t* d_stick_col = nullptr;
  int32_t* d_stick_y = nullptr;
  int32_t* d_col_x = nullptr;
  int32_t* d_stick_at = nullptr;   // ncols x n2: stick of (column, y grid index), -1 if none
  int16_t* d_xcol = nullptr;       // n1: column of each x grid index, -1 if none
  FftPlan plan[3];
  double2* d_tw64 = nullptr;        // twiddle tables, FP64
  float2* d_tw32 = nullptr;         // same, rounded to FP32
  float4* d_twdf = nullptr;         // same as double-float pairs (re.hi, re.lo, im.hi, im.lo)
  int16_t* d_perm = nullptr;        // digit-reversal tables
  int32_t* d_shell = nullptr;       // shell of each internal plane wave
  double* d_Tshell = nullptr;       // nshell kinetic energies

  // potential (internal layout [i3][i2][i1], scaled by 1/(N1 N2 N3))
  bool have_v = false;
  double vbar = 0.0;                // mean of V_LOC(r) over the grid
  double* d_v64 = nullptr;
  float* d_v32 = nullptr;
  float2* d_vdf = nullptr;          // V as double-float pairs (hi, lo)

  // projectors (internal plane-wave order, column-major ld = npw)
  int nproj = 0;
  bool d_diag = true;
  double2* d_beta64 = nullptr;
  double* d_ddiag = nullptr;        // nproj
  double2* d_dfull = nullptr;       // nproj x nproj
  float2* d_beta32 = nullptr;       // FP32 copy (mixed mode)
  void* d_beta_bf16 = nullptr;      // BF16 planar copies for the tensor-core GEMMs
  void* d_beta_bf16_t = nullptr;

  // real bands at k = 0 (gamma.cu): the half sphere in public order, the
  // internal positions of G and -G for each of its plane waves, and whether
  // the projectors keep real functions real (-1: not checked since they were set)
  std::vector<int32_t> gam_pub;
  int32_t* d_gam_pos = nullptr;
  int32_t* d_gam_neg = nullptr;
  int32_t* d_gam_shell = nullptr;   // shell of each half-sphere plane wave
  double* d_gam_kin = nullptr;      // its kinetic energy
  int64_t gam_g0 = -1;              // position of G = 0 in the half sphere
  int gam_proj_ok = -1;

  // exact exchange and ACE (exx.cu): the full-box index of each public plane
  // wave, the Coulomb factor 4 pi / (|G|^2 Omega N^3) on the box (0 at G = 0),
  // and the ACE projectors zeta (internal order, npw x ace_n; the operator is
  // -zeta zeta^H, added to H when ace_n > 0) with whether they are real
  // functions at k = 0 (-1: not checked)
  int32_t* d_boxidx = nullptr;
  double* d_kern = nullptr;
  double2* d_ace = nullptr;
  int ace_n = 0;
  int ace_real = -1;
  DevBuf<char> ws_ace;              // zeta^H psi of the ACE term (ace_n x nb)

  // overlap operator S = 1 + sum_ij |beta_i> q_ij <beta_j| of ultrasoft / PAW
  // projectors (overlap.cu): q and the separable S^-1/2 = 1 + beta K beta^H
  // (both nproj x nproj, complex FP64, column-major); with an overlap set the
  // eigensolvers solve H x = e S x
  bool have_overlap = false;
  double2* d_q = nullptr;
  double2* d_ksq = nullptr;
  DevBuf<char> ws_ov;               // products of the S and S^-1/2 applications

  // workspaces (grown on demand)
  DevBuf<char> ws_fft, ws_psi, ws_hpsi, ws_becp, ws_split, ws_host;
  DevBuf<char> ws_vnl;              // FP32 nonlocal term of the mixed H (npw x nb)
  DevBuf<char> ws_grid;             // SCF steps: a real and a complex full-box grid
  DevBuf<char> ws_tune;             // scratch of the tile autotuner
  DevBuf<char> ws_tc;               // packed BF16 operands of the tensor-core path
  DevBuf<char> ws_oz;               // sliced operands and partials of the FP64-equivalent GEMM
  int tc_nb_cap = 0, tc_P = -1;     // geometry the ws_tc zero padding was laid out for
  int* d_err = nullptr;             // device error word (bounded waits that gave up)
  float* d_mlp = nullptr;           // learned-preconditioner parameters
  bool have_mlp = false;
  DavWs* dav = nullptr;             // eigensolver workspace
  KernelTimer timer;
  int fft_batch = 32;               // bands per FFT batch (bounded by workspace)

  ~System();
};

template <typename T> void ensure(DevBuf<T>& b, size_t n) {
  if (b.n >= n) return;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.n = 0;
  PWH_CUDA(cudaMalloc((void**)&b.p, n * sizeof(T)));
  b.n = n;
}

// Brackets the launches of one kernel family with events when timing is on.
struct TimedScope {
  System& s;
  int fam;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  bool counted = false;
  TimedScope(System& s_, int fam_, cudaStream_t st_, double flops = 0, double bytes = 0)
      : s(s_), fam(fam_), st(st_) {
    if (s.timer.on) {
      counted = true;
      if (s.timer.depth++ == 0) {
        a = s.timer.get();
        cudaEventRecord(a, st);
        s.timer.flops[fam] += flops;
        s.timer.bytes[fam] += bytes;
      }
    }
  }
  ~TimedScope() {
    if (counted) --s.timer.depth;
    if (a) {
      cudaEvent_t b = s.timer.get();
      cudaEventRecord(b, st);
      s.timer.pending.push_back({fam, a, b});
    }
  }
};

// --------------------------------------------------------- entry helpers ----
template <typename F> pwh_status guarded(F&& f) {
  try {
    f();
    return PWH_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.st;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return PWH_ERR_OOM;
  } catch (...) {
    set_error("unknown internal error");
    return PWH_ERR_CUDA;
  }
}

// internal launchers (defined in the .cu files)
void build_fft_plans(System& s);
// hpsi = (kinetic + local) psi [+ vnl, an FP32 nonlocal term in the same
// layout, ld ldv, when given]
template <typename T>
void local_kinetic(System& s, int nb, const double2* psi, int64_t ldp, double2* hpsi,
                   int64_t ldh, cudaStream_t st, const float2* vnl = nullptr, int64_t ldv = 0);
void nonlocal_fp64(System& s, int nb, const double2* psi, int64_t ldp, double2* hpsi,
                   int64_t ldh, cudaStream_t st);
// vnl (FP32, ld ldv) = sum_ij beta_i D_ij <beta_j|psi> on the BF16 tensor cores
void nonlocal_mixed(System& s, int nb, const double2* psi, int64_t ldp, float2* vnl,
                    int64_t ldv, cudaStream_t st, int terms);
int* device_error_word(System& s);
void apply_internal(System& s, int nb, const double2* psi, int64_t ldp, double2* hpsi,
                    int64_t ldh, int precision);
void permute_public_to_internal(System& s, const double2* src, double2* dst, int nb,
                                int64_t lds = 0);
// rho_int ([i3][i2][i1], unscaled) += sum_b occ_b |psi_b(r)|^2 for bands in
// internal order (ld npw), occ on the device.
void density_accumulate(System& s, int nb, const double2* psi_int, const double* occ_dev,
                        double* rho_int);
// In-place unscaled 3D FFT of the full box (complex FP64, C order i3 fastest):
// forward exp(-i G.r), inverse exp(+i G.r).
// 3D FFT of nbox full boxes (complex FP64, C order, i3 fastest), bstride
// elements apart; forward exp(-i) or inverse exp(+i), both unscaled.
void box_fft(System& s, double2* box, bool inverse, int nbox = 1, int64_t bstride = 0);
// Real bands at k = 0 (gamma.cu): build the half-sphere tables and check the
// projectors (throws PWH_ERR_ARG where real bands do not apply); H on nb
// half-sphere bands, two per complex band of the full sphere.  scaled0: the
// bands store c(0) / sqrt 2 (the solver's storage, in which the real inner
// product is 2 Re of the complex one over the half sphere).
void gamma_prepare(System& s);
void gamma_apply(System& s, int nb, const double2* psi, int64_t ldp, double2* hpsi, int64_t ldh,
                 int precision, bool scaled0);

void mlp_factors(System& s, const int* idx, int k, const double* theta, const double* rn,
                 const double* eref, float* out, cudaStream_t st);

}  // namespace pwh

struct pwh_system {
  pwh::System s;
};
