// C-ABI entry points and host orchestration of the IE forward model (include/ie.h).
//
// Solve structure (Algorithm 1 of the paper with FP64 iterative refinement):
//   E := E0;  R := E0 - (I - G dsigma) E in FP64 on the whole grid;  e := |R| / |E0|     (eq. 9)
//   while e > tol:
//     for each sub-domain i (Gauss-Seidel order, or all from the same R for Jacobi):
//       b_i = R_i + A_ii E_i is the block right-hand side of eqs. 21/23, so GMRES(A_ii, b_i,
//       x0 = E_i, tol_i) is run in correction form: delta = GMRES(A_ii, R_i, x0 = 0,
//       tol_i |b_i| / |R_i|), E_i += delta (identical Krylov iterates);
//       Gauss-Seidel: R_j += G^(ji) dsigma_i delta for the later blocks j > i (interaction update)
//     R := E0 - (I - G dsigma) E in FP64; e := |R| / |E0|
// With IE_PREC_MIXED the block GMRES runs on complex64 vectors with complex64 FFT convolutions and
// the FP64 residual carries the accuracy; with IE_PREC_FP64 everything is complex128.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstddef>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "conv.cuh"
#include "green.cuh"
#include "ie.h"

namespace ie {

static const double kMu0 = 4.0e-7 * M_PI;

static int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Host-side fault injection (ie_debug_fail_allocation): when this count reaches zero the next device
// allocation reports out-of-memory without calling cudaMalloc, so the error paths can be tested without
// exhausting a GPU. Negative: off.
std::atomic<int> g_alloc_fail_countdown{-1};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t ensure(size_t b) {
    if (b <= bytes && p) return cudaSuccess;
    release();
    if (g_alloc_fail_countdown.load() >= 0 && g_alloc_fail_countdown.fetch_sub(1) == 0)
      return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = b;
    return cudaSuccess;
  }
  template <typename X> X* as() const { return reinterpret_cast<X*>(p); }
};

struct SpecSet {
  int nz_set = 0, Lz = 0;
  DevBuf G64, G32, Gdf;  // octants, 6 components: complex128, complex64, double-float
};

// Launches recorded while a CUDA graph is captured: (kernel class, algorithmic bytes) per launch, so
// the accounting can be replayed for the steps the graph actually ran.
using Tape = std::vector<std::pair<int, double>>;

// One instantiated GMRES graph (see gmres_graph) and everything its kernel arguments point at.
struct GmGraph {
  std::vector<const void*> key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  Tape pre, head, tail;
  std::vector<Tape> step;
  ~GmGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

}  // namespace ie

using namespace ie;

struct ie_ctx {
  int dev = 0;  // the CUDA device the context was created on (every call runs there)
  int nx = 0, ny = 0, nz = 0;
  long N = 0;
  double origin[3] = {0, 0, 0};
  double h = 0, sigma0 = 0, freq = 0, omega = 0;
  double2 k0{}, self{};
  int Lx = 0, Ly = 0;
  cudaStream_t stream = nullptr;
  std::string err;

  DevBuf tw64, tw32, twdf;
  DevBuf ds64, ds32, s6_stage;
  DevBuf ck64, cm64, ck32, cm32;  // contraction form: K = dsigma M and M (built on first use)
  DevBuf plane_act;               // per z plane: any non-zero contrast (device)
  std::vector<char> active;       // the same on the host
  std::vector<std::pair<int, int>> e_slabs;  // z ranges over which e is measured (empty: the whole grid)
  bool contract_ready = false;
  DevBuf cw32, cw64;             // w = M x of the contraction operator (block-local scratch)
  // GMRES as CUDA graphs: capture streams, device state, instantiated graphs (most recent last)
  cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
  DevBuf gm_state;
  std::vector<GmGraph*> gm_graphs;
  Tape* tape = nullptr;  // non-null while a graph is being captured
  bool has_contrast = false;
  std::vector<SpecSet*> specs;
  // Concurrent block-Jacobi solves (ie_opts.concurrent_blocks): one worker context per sub-domain, holding
  // that slab's contrast, its own stream and Krylov/FFT workspaces, and the parent's spectra for the
  // slab height (borrowed, not owned). Built for a split and reused while the split stays the same.
  std::vector<ie_ctx*> workers;
  std::vector<int> worker_split;
  long contrast_version = 0, worker_contrast_version = -1;
  std::vector<SpecSet*> borrowed;  // spectra owned by the parent context (workers only)
  bool owns_stream = false;        // workers create their own non-blocking stream

  DevBuf A32, B32, A64, B64;  // convolution workspaces
  long zcap32 = 0, zcap64 = 0;

  DevBuf E, E0, R;  // c128 whole-grid fields
  DevBuf Ec64;      // complex64 copy of E for the early, complex64 residuals
  DevBuf AEb;       // complex64 A_ii E_i of every block (block right-hand-side norms; see solve_one)
  DevBuf FV, FZ, PR, PZ;  // outer flexible GMRES: Arnoldi basis, preconditioned vectors, sweep input/output
  DevBuf FW32;            // its complex64 combination Z y
  bool has_field = false;
  DevBuf Einit;           // initial guess for the next solve (ie_set_initial_field_dev)
  bool has_init = false;

  // Krylov workspace (one precision at a time; sized on demand)
  DevBuf V, kx, kb, kt1, kt2;
  DevBuf part, counters, dh, dh2, dnrm, dy, flag, rxdev, Hdev, rxpart;
  double2* hpin = nullptr;  // pinned host scratch for small reductions
  int* kerr = nullptr;      // mapped pinned flag: a kernel's bounded wait gave up (checked at every sync)

  struct Prof {  // launch accounting (ie_profile_enable / ie_profile_read)
    bool on = false;
    int64_t launches[IE_K_COUNT] = {};
    double ms[IE_K_COUNT] = {}, bytes[IE_K_COUNT] = {};
    std::vector<cudaEvent_t> ev;  // event pairs, reused
    std::vector<int> cls;
    size_t used = 0;
  } prof;

  ~ie_ctx() {
    for (auto* w : workers) delete w;
    if (owns_stream && stream) {
      cudaStreamSynchronize(stream);
      cudaStreamDestroy(stream);
    }
    for (auto* g : gm_graphs) delete g;
    for (auto st : cap)
      if (st) cudaStreamDestroy(st);
    for (auto* s : specs) delete s;
    if (hpin) cudaFreeHost(hpin);
    if (kerr) cudaFreeHost(kerr);
    for (auto e : prof.ev) cudaEventDestroy(e);
  }
};

namespace {

ie_status fail(ie_ctx* c, ie_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

// Makes the context's device current for the duration of one library call and gives the calling
// thread its own current device back afterwards, so a context works whichever device the caller has
// selected (its buffers, streams and the no-allocation scratch all belong to that device).
struct DevGuard {
  int prev = -1;
  bool ok = true;
  explicit DevGuard(const ie_ctx* c) {
    if (!c) return;
    if (cudaGetDevice(&prev) != cudaSuccess) {
      prev = -1;
      ok = false;
      return;
    }
    if (prev == c->dev) {
      prev = -1;  // nothing to restore
    } else if (cudaSetDevice(c->dev) != cudaSuccess) {
      ok = false;
    }
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DevGuard(const DevGuard&) = delete;
  DevGuard& operator=(const DevGuard&) = delete;
};
#define IE_ON_CTX_DEVICE(c)                                                          \
  DevGuard ie_dev_guard_(c);                                                         \
  if (!ie_dev_guard_.ok) return fail(const_cast<ie_ctx*>(c), IE_ECUDA, "cannot make the context's device current")

#define CK(expr)                                                                              \
  do {                                                                                        \
    cudaError_t _e = (expr);                                                                  \
    if (_e != cudaSuccess)                                                                    \
      return fail(c, _e == cudaErrorMemoryAllocation ? IE_ENOMEM : IE_ECUDA,                  \
                  std::string(#expr) + ": " + cudaGetErrorString(_e));                        \
  } while (0)

#define CKS(expr)                 \
  do {                            \
    ie_status _s = (expr);        \
    if (_s != IE_OK) return _s;   \
  } while (0)

// Launch with accounting: counts the launch and its algorithmic bytes in class `cls` and, when timing
// is on, brackets it with a pair of CUDA events on the context stream.
template <class F> cudaError_t kl(ie_ctx* c, int cls, double bytes, F&& f) {
  if (c->tape) {  // inside a graph capture: record, count later per executed step
    c->tape->emplace_back(cls, bytes);
    return f();
  }
  auto& P = c->prof;
  P.launches[cls]++;
  P.bytes[cls] += bytes;
  if (!P.on) return f();
  if (2 * P.used + 2 > P.ev.size()) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) return e;
    P.ev.push_back(a);
    P.ev.push_back(b);
    P.cls.push_back(0);
  }
  cudaEvent_t a = P.ev[2 * P.used], b = P.ev[2 * P.used + 1];
  cudaError_t e = cudaEventRecord(a, c->stream);
  if (e == cudaSuccess) e = f();
  if (e == cudaSuccess) e = cudaEventRecord(b, c->stream);
  if (e == cudaSuccess) P.cls[P.used++] = cls;
  return e;
}
#define KL(cls, bytes, expr) CK(kl(c, (cls), (double)(bytes), [&]() -> cudaError_t { return (expr); }))

// Fold completed event pairs into the per-class times (call only after the stream has drained).
cudaError_t drain(ie_ctx* c) {
  auto& P = c->prof;
  for (size_t k = 0; k < P.used; ++k) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(P.ev[2 * k + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, P.ev[2 * k], P.ev[2 * k + 1]);
    if (e != cudaSuccess) return e;
    P.ms[P.cls[k]] += ms;
  }
  P.used = 0;
  return cudaSuccess;
}
cudaError_t sync(ie_ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess && c->kerr && *reinterpret_cast<volatile int*>(c->kerr)) {
    *c->kerr = 0;
    return cudaErrorLaunchTimeout;  // a staging wait in a kernel reached its spin limit
  }
  return e == cudaSuccess ? drain(c) : e;
}

// pass classes: complex64 kernels, or FP64-accurate kernels (complex128 or double-float)
template <typename T> constexpr int cls_base() { return std::is_same<T, float>::value ? IE_K_P1_C64 : IE_K_P1_C128; }

template <typename T> const C<T>* twid(const ie_ctx* c);
template <> const float2* twid<float>(const ie_ctx* c) { return c->tw32.as<float2>(); }
template <> const double2* twid<double>(const ie_ctx* c) { return c->tw64.as<double2>(); }
template <> const dfc* twid<df>(const ie_ctx* c) { return c->twdf.as<dfc>(); }
template <typename T> const FieldR<T>* dsig(const ie_ctx* c);
template <> const float* dsig<float>(const ie_ctx* c) { return c->ds32.as<float>(); }
template <> const double* dsig<double>(const ie_ctx* c) { return c->ds64.as<double>(); }
template <> const double* dsig<df>(const ie_ctx* c) { return c->ds64.as<double>(); }
template <typename T> const C<T>* spec(const SpecSet* s);
template <> const float2* spec<float>(const SpecSet* s) { return s->G32.as<float2>(); }
template <> const double2* spec<double>(const SpecSet* s) { return s->G64.as<double2>(); }
template <> const dfc* spec<df>(const SpecSet* s) { return s->Gdf.as<dfc>(); }

// Green spectra for a slab of nz_set cells: FP64 tabulation -> FP64 3D FFT -> scaled octants.
ie_status get_spec(ie_ctx* c, int nz_set, SpecSet** out) {
  for (auto* s : c->borrowed)
    if (s->nz_set == nz_set) {
      *out = s;
      return IE_OK;
    }
  for (auto* s : c->specs)
    if (s->nz_set == nz_set) {
      *out = s;
      return IE_OK;
    }
  const int Lz = next_pow2(2 * nz_set);
  if (!supported_pencil(Lz)) return fail(c, IE_EINVAL, "padded z length above 1024");
  auto* S = new SpecSet();
  S->nz_set = nz_set;
  S->Lz = Lz;
  const long ox = c->Lx / 2 + 1, oy = c->Ly / 2 + 1, oz = Lz / 2 + 1, ocs = ox * oy * oz;
  cudaError_t e1 = S->G64.ensure(sizeof(double2) * 6 * ocs);
  cudaError_t e2 = e1 == cudaSuccess ? S->G32.ensure(sizeof(float2) * 6 * ocs) : e1;
  if (e2 == cudaSuccess) e2 = S->Gdf.ensure(sizeof(dfc) * 6 * ocs);
  DevBuf full;
  cudaError_t e3 = e2 == cudaSuccess ? full.ensure(sizeof(double2) * (size_t)Lz * c->Ly * c->Lx) : e2;
  if (e3 != cudaSuccess) {
    delete S;
    return fail(c, IE_ENOMEM, "allocating Green spectra");
  }
  const double scale = 1.0 / ((double)c->Lx * c->Ly * Lz);
  double2* F = full.as<double2>();
  const double2* tw = c->tw64.as<double2>();
  for (int comp = 0; comp < 6; ++comp) {
    const double vol = (double)Lz * c->Ly * c->Lx;
    cudaError_t e = kl(c, IE_K_SETUP, 16.0 * vol, [&]() {
      return launch_green_tab(F, comp, c->Lx, c->Ly, Lz, c->nx, c->ny, nz_set, c->h, c->k0, c->sigma0, c->self,
                              c->stream);
    });
    if (e == cudaSuccess)
      e = kl(c, IE_K_SETUP, 32.0 * vol,
             [&]() { return ConvLaunch<double>::rows(c->Lx, -1, F, (long)Lz * c->Ly, tw, c->stream); });
    if (e == cudaSuccess)  // y: element e of lane x in plane z at z*Ly*Lx + e*Lx + x
      e = kl(c, IE_K_SETUP, 32.0 * vol, [&]() {
        return ConvLaunch<double>::lanes(c->Ly, -1, 0, F, 0, (long)c->Ly * c->Lx, c->Lx, c->Ly, F, 0,
                                         (long)c->Ly * c->Lx, c->Lx, c->Ly, c->Lx, Lz, 1, tw, c->stream);
      });
    if (e == cudaSuccess)  // z: element e of lane x in row y at y*Lx + e*Ly*Lx + x
      e = kl(c, IE_K_SETUP, 32.0 * vol, [&]() {
        return ConvLaunch<double>::lanes(Lz, -1, 0, F, 0, c->Lx, (long)c->Ly * c->Lx, Lz, F, 0, c->Lx,
                                         (long)c->Ly * c->Lx, Lz, c->Lx, c->Ly, 1, tw, c->stream);
      });
    if (e == cudaSuccess)
      e = kl(c, IE_K_SETUP, 16.0 * ocs + 24.0 * ocs, [&]() {
        return launch_extract_octant(F, c->Lx, c->Ly, Lz, scale, S->G64.as<double2>() + comp * ocs,
                                     S->G32.as<float2>() + comp * ocs, S->Gdf.as<dfc>() + comp * ocs, c->stream);
      });
    if (e != cudaSuccess) {
      delete S;
      return fail(c, IE_ECUDA, std::string("Green spectra: ") + cudaGetErrorString(e));
    }
  }
  cudaError_t e = sync(c);  // `full` is freed on return
  if (e != cudaSuccess) {
    delete S;
    return fail(c, IE_ECUDA, std::string("Green spectra: ") + cudaGetErrorString(e));
  }
  c->specs.push_back(S);
  *out = S;
  return IE_OK;
}

// complex64 workspaces for float; the 16-byte complex128 / double-float kernels share the others
template <typename T> ie_status ensure_conv_ws(ie_ctx* c, int zcap) {
  long& cap = std::is_same<T, float>::value ? c->zcap32 : c->zcap64;
  DevBuf& A = std::is_same<T, float>::value ? c->A32 : c->A64;
  DevBuf& B = std::is_same<T, float>::value ? c->B32 : c->B64;
  if (zcap <= cap) return IE_OK;
  CK(A.ensure(sizeof(C<T>) * 3 * (size_t)zcap * c->ny * c->Lx));
  CK(B.ensure(sizeof(C<T>) * 3 * (size_t)zcap * c->Ly * c->Lx));
  cap = zcap;
  return IE_OK;
}

// ------------------------------------------------------------------ FFT tile autotuner
// The strided passes (P2, P3, P4) have three tile shapes: the default, one with half the pencils per
// block and one with twice as many (P3 a fourth with four times as many); P3 has each also with TMA
// staging of its input pencils, and its two widest tiles also with mirrored rows (twelve variants,
// of which a precision may build fewer). The first convolution
// of a new shape times every variant on the live buffers
// (three timed launches each after a warm-up; the work is data independent) and keeps the fastest for
// the rest of the process. Variants produce bit-identical results.
struct TuneKey {
  int kind, bytes, L, Lx, Ly, nz, nz2;
  bool operator<(const TuneKey& o) const {
    return std::tie(kind, bytes, L, Lx, Ly, nz, nz2) < std::tie(o.kind, o.bytes, o.L, o.Lx, o.Ly, o.nz, o.nz2);
  }
};
std::map<TuneKey, int> g_tuned;
std::map<TuneKey, std::vector<float>> g_tune_ms;  // mean time of one launch of each variant (ms)
std::mutex g_tune_mu;

// Tile variant forced for a pass kind (2 = P2, 3 = P3, 4 = P4) by ie_debug_force_tile; -1: autotuned.
std::atomic<int> g_force_tile[5] = {{-1}, {-1}, {-1}, {-1}, {-1}};

int tuned_variant(const TuneKey& k) {
  if (k.kind >= 2 && k.kind <= 4) {
    const int f = g_force_tile[k.kind].load();
    if (f >= 0) return f;
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(k);
  return it == g_tuned.end() ? -1 : it->second;
}

// Time each variant of one launch (run(v) enqueues it on the context stream) and record the fastest.
template <class F> cudaError_t tune(ie_ctx* c, const TuneKey& k, F&& run, int* best, int nvar = kTileVariants) {
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  float best_ms = 1e30f;
  *best = 0;
  std::vector<float> times;
  for (int v = 0; v < nvar && e == cudaSuccess; ++v) {
    e = run(v);  // warm-up (module load, caches)
    if (e == cudaErrorNotSupported) {  // a tile this arithmetic does not build: nothing was launched
      e = cudaSuccess;
      times.push_back(INFINITY);
      continue;
    }
    if (e == cudaSuccess) e = cudaEventRecord(a, c->stream);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = run(v);
    if (e == cudaSuccess) e = cudaEventRecord(b, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    times.push_back(ms / 3.f);
    if (e == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      *best = v;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[k] = *best;
    g_tune_ms[k] = times;
  }
  return e;
}

// One FFT convolution G^(ts) dsigma^(s) x with the given spectra and epilogue (see conv_kernels.cuh).
//   x: source field, components at stride x_cs, covering the slab [zs0, zs0 + nzs) of the grid;
//   os/ot: pencil positions of the source / target slab inside the padded z axis of `S`.
// Contraction form of P1 (see k_p1_contrast_fftx): K = dsigma M and M on the whole grid, w the
// block-local destination of M x.
template <typename T> struct Contract {
  const FieldR<T>* K;
  const FieldR<T>* M;
  FieldC<T>* w;
  long w_cs;
};

template <typename T>
ie_status conv(ie_ctx* c, const SpecSet* S, const FieldC<T>* x, long x_cs, int zs0, int nzs, int os, int nzt, int ot,
               int mode, const FieldC<T>* xin, long xin_cs, FieldC<T>* y, long y_cs, double2* r, long r_cs,
               const double2* b, long b_cs, const Contract<T>* ca = nullptr) {
  CKS(ensure_conv_ws<T>(c, std::max(nzs, nzt)));
  const long zc = std::is_same<T, float>::value ? c->zcap32 : c->zcap64;
  C<T>* A = (std::is_same<T, float>::value ? c->A32 : c->A64).template as<C<T>>();
  C<T>* B = (std::is_same<T, float>::value ? c->B32 : c->B64).template as<C<T>>();
  const long A_cs = zc * c->ny * c->Lx, B_cs = zc * c->Ly * c->Lx;
  const long nxy = (long)c->nx * c->ny;
  const C<T>* tw = twid<T>(c);
  cudaStream_t s = c->stream;
  // algorithmic bytes of the pass model: every pass reads and writes its operands exactly once
  const double sz = sizeof(C<T>), ocs = (double)(c->Lx / 2 + 1) * (c->Ly / 2 + 1) * (S->Lz / 2 + 1);
  const double fz = sizeof(FieldC<T>), rz = sizeof(FieldR<T>);
  const double epi = mode == EPI_APPLY ? 2 * fz : mode == EPI_CONV ? fz : mode == EPI_ACCUM128 ? 32.0 : 32.0 + fz;
  const int k0 = cls_base<T>();
  const int bz = (int)sizeof(C<T>) + (std::is_same<T, df>::value ? 1 : 0);  // tells the three arithmetics apart
  const TuneKey k2{2, bz, c->Ly, c->Lx, c->ny, nzs, 0}, k3{3, bz, S->Lz, c->Lx, c->Ly, nzs, nzt},
      k4{4, bz, c->Ly, c->Lx, c->ny, nzt, 0};
  auto p1 = [&]() {
    if (ca)
      return ConvLaunch<T>::p1(c->Lx, x, x_cs, ca->K + (long)zs0 * nxy, c->N, A, A_cs, c->nx, (long)nzs * c->ny, tw, s,
                               ca->M + (long)zs0 * nxy, ca->w, ca->w_cs);
    return ConvLaunch<T>::p1(c->Lx, x, x_cs, dsig<T>(c) + (long)zs0 * nxy, c->N, A, A_cs, c->nx, (long)nzs * c->ny, tw,
                             s);
  };
  auto p2 = [&](int v) {
    return ConvLaunch<T>::lanes(c->Ly, -1, v, A, A_cs, (long)c->ny * c->Lx, c->Lx, c->ny, B, B_cs, (long)c->Ly * c->Lx,
                                c->Lx, c->Ly, c->Lx, nzs, 3, tw, s);
  };
  auto p3 = [&](int v) {
    return ConvLaunch<T>::p3(S->Lz, v, B, B_cs, nzs, os, B, B_cs, nzt, ot, spec<T>(S), c->Lx, c->Ly, tw, c->kerr, s);
  };
  auto p4 = [&](int v) {
    return ConvLaunch<T>::lanes(c->Ly, +1, v, B, B_cs, (long)c->Ly * c->Lx, c->Lx, c->Ly, A, A_cs, (long)c->ny * c->Lx,
                                c->Lx, c->ny, c->Lx, nzt, 3, tw, s);
  };
  KL(k0 + 0, (3 * fz + 6 * rz + (ca ? 6 * rz + 3 * fz : 0.0)) * nzs * nxy + 3 * sz * nzs * c->ny * c->Lx, p1());
  int v2 = tuned_variant(k2), v3 = tuned_variant(k3), v4 = tuned_variant(k4);
  if (v2 < 0) CK(tune(c, k2, p2, &v2));
  KL(k0 + 1, 3 * sz * nzs * c->Lx * (double)(c->ny + c->Ly), p2(v2));
  if (v3 < 0) {  // P3 works in place: tune on the live B, then rebuild B from x before the real pass
    CK(tune(c, k3, p3, &v3, kP3TileVariants));
    CK(p1());
    CK(p2(v2));
  }
  KL(k0 + 2, 3 * sz * (double)(nzs + nzt) * c->Ly * c->Lx + 6 * sz * ocs, p3(v3));
  if (v4 < 0) CK(tune(c, k4, p4, &v4));
  KL(k0 + 3, 3 * sz * nzt * c->Lx * (double)(c->Ly + c->ny), p4(v4));
  KL(k0 + 4, 3 * sz * nzt * c->ny * c->Lx + 3 * epi * nzt * nxy,
     ConvLaunch<T>::p5(c->Lx, mode, A, A_cs, c->nx, (long)nzt * c->ny, xin, xin_cs, y, y_cs, r, r_cs, b, b_cs, tw, s));
  return IE_OK;
}

// Operator of one sub-domain, y = (I - G^(ii) dsigma^(i)) x, on block-local vectors.
template <typename T> const FieldR<T>* ctens(const ie_ctx* c, bool k);
template <> const float* ctens<float>(const ie_ctx* c, bool k) { return (k ? c->ck32 : c->cm32).as<float>(); }
template <> const double* ctens<double>(const ie_ctx* c, bool k) { return (k ? c->ck64 : c->cm64).as<double>(); }
template <> const double* ctens<df>(const ie_ctx*, bool) { return nullptr; }

// Tensors of the contraction form for the current contrast (built once per ie_set_contrast).
ie_status ensure_contract(ie_ctx* c) {
  if (c->contract_ready) return IE_OK;
  CK(c->ck64.ensure(sizeof(double) * 6 * c->N));
  CK(c->cm64.ensure(sizeof(double) * 6 * c->N));
  CK(c->ck32.ensure(sizeof(float) * 6 * c->N));
  CK(c->cm32.ensure(sizeof(float) * 6 * c->N));
  KL(IE_K_FIELD, 144.0 * c->N,
     launch_contract_tensors(c->ds64.as<double>(), c->N, c->sigma0, c->ck64.as<double>(), c->cm64.as<double>(),
                             c->ck32.as<float>(), c->cm32.as<float>(), c->stream));
  c->contract_ready = true;
  return IE_OK;
}

// Operator of one sub-domain on block-local vectors: y = (I - G^(ii) dsigma^(i)) x (eq. 8 restricted to
// the slab), or with `contract` the contraction form y = (M - G^(ii) dsigma^(i) M) x, the same operator
// right-multiplied by M = 2 sigma0 (sigma + sigma0 I)^-1 (apply_conv always gives the first).
template <typename T> struct BlockOp {
  ie_ctx* c;
  int z0, nz;
  const SpecSet* S;
  bool contract = false;
  long nb() const { return (long)nz * c->ny * c->nx; }
  ie_status apply_conv(const FieldC<T>* x, FieldC<T>* y) const {
    return conv<T>(c, S, x, nb(), z0, nz, 0, nz, 0, EPI_APPLY, x, nb(), y, nb(), nullptr, 0, nullptr, 0);
  }
  ie_status apply(const FieldC<T>* x, FieldC<T>* y) const {
    if (!contract) return apply_conv(x, y);
    DevBuf& wb = std::is_same<T, float>::value ? c->cw32 : c->cw64;
    CK(wb.ensure(sizeof(FieldC<T>) * 3 * nb()));
    FieldC<T>* w = wb.template as<FieldC<T>>();
    const Contract<T> ca{ctens<T>(c, true), ctens<T>(c, false), w, nb()};
    return conv<T>(c, S, x, nb(), z0, nz, 0, nz, 0, EPI_APPLY, w, nb(), y, nb(), nullptr, 0, nullptr, 0, &ca);
  }
  // x := M x (turns the contraction-form solution into the field correction)
  ie_status to_field(FieldC<T>* x) const {
    if (!contract) return IE_OK;
    const long nxy = (long)c->nx * c->ny;
    KL(IE_K_FIELD, (6.0 * sizeof(FieldR<T>) + 6.0 * sizeof(FieldC<T>)) * nb(),
       launch_apply_sym6(ctens<T>(c, false) + (long)z0 * nxy, c->N, x, nb(), nb(), c->stream));
    return IE_OK;
  }
};

template <typename T> ie_status make_block(ie_ctx* c, int z0, int nz, BlockOp<T>* op, bool contract = false) {
  if (z0 < 0 || nz < 1 || z0 + nz > c->nz) return fail(c, IE_EINVAL, "slab outside the grid");
  if (!c->has_contrast) return fail(c, IE_ESTATE, "no contrast set");
  if (contract && std::is_same<T, df>::value) return fail(c, IE_EINVAL, "contraction form: complex64 or complex128");
  SpecSet* S = nullptr;
  CKS(get_spec(c, nz, &S));
  if (contract) CKS(ensure_contract(c));
  *op = BlockOp<T>{c, z0, nz, S, contract};
  return IE_OK;
}

// Worker context for the slab [z0, z0 + nz) of c (concurrent block-Jacobi solves): the same cell size,
// background and frequency on a grid of nz planes, its own non-blocking stream, error flag and
// workspaces, and the parent's spectra for the slab height. Its twiddles and contrast are copied from
// the parent on the parent's stream (prepare_workers orders the worker streams after those copies).
ie_status make_worker(ie_ctx* c, int z0, int nz, ie_ctx** out) {
  *out = nullptr;
  SpecSet* S = nullptr;
  CKS(get_spec(c, nz, &S));
  auto* w = new (std::nothrow) ie_ctx();
  if (!w) return fail(c, IE_ENOMEM, "allocating a worker context");
  w->dev = c->dev;
  w->nx = c->nx;
  w->ny = c->ny;
  w->nz = nz;
  w->N = (long)nz * c->nx * c->ny;
  for (int a = 0; a < 3; ++a) w->origin[a] = c->origin[a];
  w->origin[2] += z0 * c->h;
  w->h = c->h;
  w->sigma0 = c->sigma0;
  w->freq = c->freq;
  w->omega = c->omega;
  w->k0 = c->k0;
  w->self = c->self;
  w->Lx = c->Lx;
  w->Ly = c->Ly;
  w->borrowed.push_back(S);
  auto bad = [&](ie_status st, const std::string& what) {
    delete w;
    return fail(c, st, what);
  };
  if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess)
    return bad(IE_ECUDA, "creating a worker stream");
  w->owns_stream = true;
  if (cudaHostAlloc(reinterpret_cast<void**>(&w->kerr), sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
    w->kerr = nullptr;
    return bad(IE_ENOMEM, "allocating a worker flag");
  }
  *w->kerr = 0;
  cudaError_t e = w->tw64.ensure(sizeof(double2) * TWN);
  if (e == cudaSuccess) e = w->tw32.ensure(sizeof(float2) * TWN);
  if (e == cudaSuccess) e = w->twdf.ensure(sizeof(dfc) * TWN);
  if (e == cudaSuccess) e = w->ds64.ensure(sizeof(double) * 6 * w->N);
  if (e == cudaSuccess) e = w->ds32.ensure(sizeof(float) * 6 * w->N);
  if (e != cudaSuccess) return bad(e == cudaErrorMemoryAllocation ? IE_ENOMEM : IE_ECUDA, "worker buffers");
  e = cudaMemcpyAsync(w->tw64.p, c->tw64.p, sizeof(double2) * TWN, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w->tw32.p, c->tw32.p, sizeof(float2) * TWN, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w->twdf.p, c->twdf.p, sizeof(dfc) * TWN, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return bad(IE_ECUDA, "copying twiddles to a worker");
  *out = w;
  return IE_OK;
}

// Worker contexts for the sub-domains of `split`, with the current contrast (copied on the parent
// stream; see order_workers).
ie_status prepare_workers(ie_ctx* c, const std::vector<int>& split) {
  const int M = (int)split.size() - 1;
  const long nxy = (long)c->nx * c->ny;
  if (c->worker_split != split) {
    for (auto* w : c->workers) delete w;
    c->workers.clear();
    c->worker_split.clear();
    std::vector<ie_ctx*> ws;
    for (int i = 0; i < M; ++i) {
      ie_ctx* w = nullptr;
      const ie_status st = make_worker(c, split[i], split[i + 1] - split[i], &w);
      if (st != IE_OK) {
        for (auto* x : ws) delete x;
        return st;
      }
      ws.push_back(w);
    }
    c->workers = ws;
    c->worker_split = split;
    c->worker_contrast_version = -1;
  }
  if (c->worker_contrast_version != c->contrast_version) {
    for (int i = 0; i < M; ++i) {
      ie_ctx* w = c->workers[i];
      const long nb = w->N, off = (long)split[i] * nxy;
      for (int k = 0; k < 6; ++k) {
        CK(cudaMemcpyAsync(w->ds64.as<double>() + k * nb, c->ds64.as<double>() + k * c->N + off, sizeof(double) * nb,
                           cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(w->ds32.as<float>() + k * nb, c->ds32.as<float>() + k * c->N + off, sizeof(float) * nb,
                           cudaMemcpyDeviceToDevice, c->stream));
      }
      w->has_contrast = true;
      w->contract_ready = false;
    }
    c->worker_contrast_version = c->contrast_version;
  }
  for (auto* w : c->workers) {
    if (w->prof.on != c->prof.on) {
      w->prof.on = c->prof.on;
      w->prof.used = 0;
    }
  }
  return IE_OK;
}

// Orders the work enqueued next on every worker stream after everything enqueued so far on the parent
// stream.
ie_status order_workers(ie_ctx* c, cudaEvent_t ev) {
  CK(cudaEventRecord(ev, c->stream));
  for (auto* w : c->workers) CK(cudaStreamWaitEvent(w->stream, ev, 0));
  return IE_OK;
}

// Adds a worker's launch accounting to its parent's and clears it (after the worker stream drained).
void fold_profile(ie_ctx* c, ie_ctx* w) {
  for (int k = 0; k < IE_K_COUNT; ++k) {
    c->prof.launches[k] += w->prof.launches[k];
    c->prof.ms[k] += w->prof.ms[k];
    c->prof.bytes[k] += w->prof.bytes[k];
    w->prof.launches[k] = 0;
    w->prof.ms[k] = 0.0;
    w->prof.bytes[k] = 0.0;
  }
}

ie_status ensure_scalars(ie_ctx* c) {
  if (!c->counters.p) {
    CK(c->counters.ensure(sizeof(unsigned) * kCounters));
    CK(cudaMemsetAsync(c->counters.p, 0, sizeof(unsigned) * kCounters, c->stream));
  }
  CK(c->part.ensure(sizeof(double2) * kRedBlocks * kRedSlots));
  CK(c->dh.ensure(sizeof(double2) * 160));
  CK(c->dh2.ensure(sizeof(double2) * 160));
  CK(c->dnrm.ensure(sizeof(double2) * 8));
  CK(c->dy.ensure(sizeof(double2) * 160));
  CK(c->flag.ensure(sizeof(int) * 4));
  if (!c->hpin) CK(cudaMallocHost(&c->hpin, sizeof(double2) * 320));
  return IE_OK;
}

RedScratch scratch(ie_ctx* c) { return RedScratch{c->part.as<double2>(), c->counters.as<unsigned>()}; }

// device FP64 scalar -> host
ie_status scalar_to_host(ie_ctx* c, const double2* dev, double2* host) {
  CK(cudaMemcpyAsync(c->hpin, dev, sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
  CK(sync(c));
  *host = c->hpin[0];
  return IE_OK;
}

template <typename T> ie_status vnorm(ie_ctx* c, const C<T>* v, long n, double* out) {
  double2* d = c->dnrm.as<double2>() + 2;
  KL(IE_K_KRYLOV_MISC, sizeof(C<T>) * (double)n, Krylov<T>::norm2(v, n, d, scratch(c), c->stream));
  double2 h;
  CKS(scalar_to_host(c, d, &h));
  *out = std::sqrt(std::max(h.x, 0.0));
  return IE_OK;
}

ie_status norm_c128(ie_ctx* c, const double2* a, long a_cs, const float2* b, long b_cs, long n, double* out) {
  double2* d = c->dnrm.as<double2>() + 3;
  KL(IE_K_FIELD, (16.0 + (b ? 8.0 : 0.0)) * 3 * n, launch_norm2_c128(a, a_cs, b, b_cs, n, d, scratch(c), c->stream));
  double2 h;
  CKS(scalar_to_host(c, d, &h));
  *out = std::sqrt(std::max(h.x, 0.0));
  return IE_OK;
}

// |a| over the z slabs of c->e_slabs (the whole grid when empty) for a whole-grid c128 field.
ie_status slab_norm(ie_ctx* c, const double2* a, double* out) {
  if (c->e_slabs.empty()) return norm_c128(c, a, c->N, nullptr, 0, c->N, out);
  const long nxy = (long)c->nx * c->ny;
  double sq = 0.0;
  for (const auto& sl : c->e_slabs) {
    double v;
    CKS(norm_c128(c, a + (long)sl.first * nxy, c->N, nullptr, 0, (long)sl.second * nxy, &v));
    sq += v * v;
  }
  *out = std::sqrt(sq);
  return IE_OK;
}

struct GmresOut {
  int iters = 0, matvecs = 0, reorth = 0;
  double rel = 0;
  bool converged = false;
};

// Restarted GMRES(m) for A x = b (Saad & Schultz). Arnoldi: classical Gram-Schmidt; for tolerances
// below kReorthTol a second pass is added whenever the projected norm drops below 1/sqrt(2) of the
// original (Daniel-Gragg-Kaufman-Stewart test, decided on the device). A loose solve (the adaptive
// sub-domain solves of Algorithm 1 ask for roughly one digit) keeps one pass: the loss of
// orthogonality of one-pass CGS in FP32 stays orders of magnitude below such a target, and the true
// residual confirms convergence at every restart. FP64 Hessenberg and Givens rotations on the host;
// stopping on the relative residual |b - A x| / |b| (eq. 9).
// x holds x0 on entry unless x0_zero. Workspace c->V holds m+1 basis vectors.
constexpr double kReorthTol = 1e-3;
// verify = false: when a cycle's Arnoldi estimate reaches tol, the solve ends there without the true
// residual (one operator application) that otherwise confirms it and leaves b - A x in c->kt1; for
// callers that use the result only as an inexact solve (the preconditioner sweeps of the outer Krylov
// iteration).
template <typename T>
ie_status gmres(ie_ctx* c, const BlockOp<T>& A, const C<T>* b, C<T>* x, bool x0_zero, double tol, int m, int max_it,
                GmresOut* out, bool verify = true) {
  const bool cgs2 = tol < kReorthTol;
  const long n = 3 * A.nb();
  cudaStream_t s = c->stream;
  CKS(ensure_scalars(c));
  if (m < 1 || m > 127) return fail(c, IE_EINVAL, "restart must be in [1, 127]");
  const long ld = (n + 1) & ~1L;  // even stride keeps every basis vector 16-byte aligned
  CK(c->V.ensure(sizeof(C<T>) * (size_t)(m + 1) * ld));
  CK(c->kt1.ensure(sizeof(C<T>) * (size_t)n));
  C<T>* V = c->V.as<C<T>>();
  C<T>* tmp = c->kt1.as<C<T>>();
  const RedScratch sc = scratch(c);
  double2* dh = c->dh.as<double2>();
  double2* dh2 = c->dh2.as<double2>();
  double2* dn = c->dnrm.as<double2>();
  int* flag = c->flag.as<int>();
  *out = GmresOut();

  double bnorm;
  CKS(vnorm<T>(c, b, n, &bnorm));
  if (bnorm == 0.0) {
    CK(cudaMemsetAsync(x, 0, sizeof(C<T>) * n, s));
    out->converged = true;
    return IE_OK;
  }
  double beta;
  if (x0_zero) {
    CK(cudaMemsetAsync(x, 0, sizeof(C<T>) * n, s));
    KL(IE_K_KRYLOV_MISC, 2.0 * sizeof(C<T>) * n, Krylov<T>::scale(b, V, n, nullptr, 1.0 / bnorm, s));
    beta = bnorm;
  } else {
    CKS(A.apply(x, tmp));
    out->matvecs++;
    KL(IE_K_KRYLOV_MISC, 3.0 * sizeof(C<T>) * n, Krylov<T>::rsub(b, tmp, n, dn + 1, sc, s));
    double2 h;
    CKS(scalar_to_host(c, dn + 1, &h));
    beta = std::sqrt(std::max(h.x, 0.0));
    if (beta / bnorm <= tol) {
      out->rel = beta / bnorm;
      out->converged = true;
      return IE_OK;
    }
    KL(IE_K_KRYLOV_MISC, 2.0 * sizeof(C<T>) * n, Krylov<T>::scale(tmp, V, n, nullptr, 1.0 / beta, s));
  }
  out->rel = beta / bnorm;
  std::vector<std::complex<double>> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  auto Hij = [&](int i, int j) -> std::complex<double>& { return H[(size_t)i * m + j]; };
  while (true) {
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jd = 0;
    bool breakdown = false;
    for (int j = 0; j < m; ++j) {
      C<T>* w = V + (size_t)(j + 1) * ld;
      CKS(A.apply(V + (size_t)j * ld, w));
      out->matvecs++;
      const int nv = j + 1;
      const double sz = sizeof(C<T>), ng = (nv + kDotGroup - 1) / kDotGroup;
      // first pass: dh[0..j] = V^H w, dh[nv] = |w|^2; w -= V dh, dn = |w|^2, flag = (|w| dropped below 1/sqrt 2)
      KL(IE_K_DOTS, sz * n * (nv + ng), Krylov<T>::dots(V, ld, nv, w, n, cgs2, dh, nullptr, nullptr, sc, s));
      KL(IE_K_UPDATE, sz * n * (nv + 2),
         Krylov<T>::update(V, ld, nv, dh, w, n, dn, dh + nv, 0.5, cgs2 ? flag : nullptr, nullptr, sc, s));
      if (cgs2) {  // second pass, launched always but run only when the flag is set (its bytes are added below)
        KL(IE_K_DOTS, 0, Krylov<T>::dots(V, ld, nv, w, n, false, dh2, dh, flag, sc, s));
        KL(IE_K_UPDATE, 0, Krylov<T>::update(V, ld, nv, dh2, w, n, dn, nullptr, 0.0, nullptr, flag, sc, s));
      }
      KL(IE_K_KRYLOV_MISC, 2 * sz * n, Krylov<T>::scale(w, w, n, dn, 0.0, s));
      CK(cudaMemcpyAsync(c->hpin, dh, sizeof(double2) * nv, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(c->hpin + nv, dn, sizeof(double2), cudaMemcpyDeviceToHost, s));
      if (cgs2) CK(cudaMemcpyAsync(c->hpin + nv + 1, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(sync(c));
      int reorth = 0;
      if (cgs2) std::memcpy(&reorth, c->hpin + nv + 1, sizeof(int));
      if (reorth) {
        c->prof.bytes[IE_K_DOTS] += sz * n * (nv + ng);
        c->prof.bytes[IE_K_UPDATE] += sz * n * (nv + 2);
        out->reorth++;
      }
      for (int i = 0; i < nv; ++i) Hij(i, j) = std::complex<double>(c->hpin[i].x, c->hpin[i].y);
      const double hn = std::sqrt(std::max(c->hpin[nv].x, 0.0));
      Hij(j + 1, j) = hn;
      for (int i = 0; i < j; ++i) {
        const std::complex<double> t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -std::conj(sn[i]) * Hij(i, j) + std::conj(cs[i]) * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      const std::complex<double> a = Hij(j, j), d = Hij(j + 1, j);
      const double den = std::sqrt(std::norm(a) + std::norm(d));
      cs[j] = den != 0.0 ? std::conj(a) / den : 1.0;
      sn[j] = den != 0.0 ? std::conj(d) / den : 0.0;
      Hij(j, j) = cs[j] * a + sn[j] * d;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -std::conj(sn[j]) * g[j];
      g[j] = cs[j] * g[j];
      out->iters++;
      jd = j + 1;
      breakdown = (hn == 0.0);
      const double est = std::abs(g[j + 1]) / bnorm;
      if (!std::isfinite(est)) return fail(c, IE_ECUDA, "GMRES produced a non-finite residual");
      if (est <= tol || breakdown || out->iters >= max_it) break;
    }
    for (int i = jd - 1; i >= 0; --i) {  // back substitution
      std::complex<double> acc = g[i];
      for (int k = i + 1; k < jd; ++k) acc -= Hij(i, k) * y[k];
      y[i] = acc / Hij(i, i);
    }
    for (int i = 0; i < jd; ++i) c->hpin[i] = make_double2(y[i].real(), y[i].imag());
    CK(cudaMemcpyAsync(c->dy.as<double2>(), c->hpin, sizeof(double2) * jd, cudaMemcpyHostToDevice, s));
    KL(IE_K_KRYLOV_MISC, sizeof(C<T>) * (double)n * (jd + 2), Krylov<T>::combine(V, ld, jd, c->dy.as<double2>(), x, n, s));
    const double est_rel = std::abs(g[jd]) / bnorm;
    if (!verify && est_rel <= tol) {
      out->rel = est_rel;
      out->converged = true;
      return IE_OK;
    }
    CKS(A.apply(x, tmp));
    out->matvecs++;
    KL(IE_K_KRYLOV_MISC, 3.0 * sizeof(C<T>) * n, Krylov<T>::rsub(b, tmp, n, dn + 1, sc, s));
    double2 h;
    CKS(scalar_to_host(c, dn + 1, &h));
    beta = std::sqrt(std::max(h.x, 0.0));
    out->rel = beta / bnorm;
    if (out->rel <= tol) {
      out->converged = true;
      return IE_OK;
    }
    if (out->iters >= max_it || beta == 0.0) return IE_OK;
    KL(IE_K_KRYLOV_MISC, 2.0 * sizeof(C<T>) * n, Krylov<T>::scale(tmp, V, n, nullptr, 1.0 / beta, s));
  }
}

ie_status check_point(ie_ctx* c, const double* p) {
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(p[a])) return fail(c, IE_EINVAL, "non-finite position");
  double d2 = 0.0;
  const int n[3] = {c->nx, c->ny, c->nz};
  bool inside = true;
  for (int a = 0; a < 3; ++a) {
    const double u = (p[a] - c->origin[a]) / c->h - 0.5;  // fractional cell index of the nearest centre
    const double k = std::round(u);
    if (k < 0 || k > n[a] - 1) inside = false;
    d2 += (u - k) * (u - k);
  }
  if (inside && std::sqrt(d2) < 1e-9) return fail(c, IE_EINVAL, "source or receiver on a cell centre");
  return IE_OK;
}

// Residuals above max(kFastResidualFloor, 10 tol) are evaluated with the complex64 kernels: their
// rounding error, about 1e-7 of |E0| + |G dsigma E|, is then at most a few per cent of e, which neither
// the adaptive block tolerance e/10 (one digit) nor the test e > tol (a margin of 10x) can notice. Every
// residual below it, and so the final convergence decision and the reported e, is FP64-accurate.
constexpr double kFastResidualFloor = 1e-5;
inline double fast_residual_above(double tol) { return std::max(kFastResidualFloor, 10.0 * tol); }

// Whole-grid residual R = E0 - (I - G dsigma) E and its relative norm e (eq. 9): FP64-accurate
// (double-float kernels), or complex64 when `fast` (recomputed FP64-accurately if e falls to
// `fast_above` or below).
ie_status full_residual(ie_ctx* c, double e0norm, double* e, bool fast = false, double fast_above = 1e-3) {
  SpecSet* S = nullptr;
  CKS(get_spec(c, c->nz, &S));
  if (fast) {
    CK(c->Ec64.ensure(sizeof(float2) * 3 * c->N));
    float2* E32 = c->Ec64.as<float2>();
    KL(IE_K_FIELD, 72.0 * c->N, launch_c128_to_c64(c->E.as<double2>(), c->N, E32, c->N, c->N, c->stream));
    CKS(conv<float>(c, S, E32, c->N, 0, c->nz, 0, c->nz, 0, EPI_RESID128, E32, c->N, nullptr, 0, c->R.as<double2>(),
                    c->N, c->E0.as<double2>(), c->N));
    double rn;
    CKS(slab_norm(c, c->R.as<double2>(), &rn));
    *e = rn / e0norm;
    if (!std::isfinite(*e)) return fail(c, IE_ECUDA, "non-finite residual");
    if (*e > fast_above) return IE_OK;
  }
  const double2* Ed = c->E.as<double2>();
  CKS(conv<df>(c, S, Ed, c->N, 0, c->nz, 0, c->nz, 0, EPI_RESID128, Ed, c->N, nullptr, 0, c->R.as<double2>(), c->N,
               c->E0.as<double2>(), c->N));
  double rn;
  CKS(slab_norm(c, c->R.as<double2>(), &rn));
  *e = rn / e0norm;
  if (!std::isfinite(*e)) return fail(c, IE_ECUDA, "non-finite residual");
  return IE_OK;
}

// ---------------------------------------------------------------- GMRES as one CUDA graph
// gmres<T> with x0 = 0, with the Givens rotations, the stopping tests and the restart decision on the
// device (krylov.cu, k_gm_*). A conditional WHILE node runs restart cycles; inside it m conditional IF
// nodes run the Arnoldi steps j = 0..m-1 (each step enables the next one unless it met the tolerance,
// broke down or reached the iteration limit, so the later steps are skipped), followed by the
// back substitution, x += V y, the true residual b - A x and the restart test. A block solve is one
// graph launch and one host synchronisation instead of one synchronisation per Arnoldi step. Every
// wait is bounded: each cycle runs at most m steps, and the WHILE condition is cleared once the
// iterations or the cycles reach max_it. Graphs are cached per block shape, restart length and the
// buffers their kernels address.
constexpr int kGmGraphCache = 8;

void account(ie_ctx* c, const Tape& t) {
  for (const auto& e : t) {
    c->prof.launches[e.first]++;
    c->prof.bytes[e.first] += e.second;
  }
}

ie_status cap_stream(ie_ctx* c, int k) {
  if (!c->cap[k]) CK(cudaStreamCreateWithFlags(&c->cap[k], cudaStreamNonBlocking));
  return IE_OK;
}

// Adds a conditional node after the current capture point of `st` and returns its body graph.
ie_status add_conditional(ie_ctx* c, cudaStream_t st, cudaGraphConditionalHandle h,
                          cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return fail(c, IE_ECUDA, "graph capture is not active");
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h;
  prm.conditional.type = type;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  const cudaError_t e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &prm);
  if (e != cudaSuccess)
    return fail(c, IE_ECUDA, std::string("adding a conditional ") + (type == cudaGraphCondTypeWhile ? "WHILE" : "IF") +
                                 " node: " + cudaGetErrorString(e));
  CK(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  *body = prm.conditional.phGraph_out[0];
  return IE_OK;
}

// Ends every capture still open on the context's capture streams (after a failed build).
void abandon_capture(ie_ctx* c) {
  for (int k = 2; k >= 0; --k) {
    if (!c->cap[k]) continue;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->cap[k], &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(c->cap[k], &g);
      if (k == 0 && g) cudaGraphDestroy(g);  // the bodies belong to their conditional nodes
    }
  }
  cudaGetLastError();
}

template <typename T>
ie_status build_gmres_graph(ie_ctx* c, const BlockOp<T>& A, const C<T>* b, C<T>* x, int m, bool cgs2, long n,
                            long ld, GmGraph* G) {
  C<T>* V = c->V.as<C<T>>();
  C<T>* tmp = c->kt1.as<C<T>>();
  GmState* st = c->gm_state.as<GmState>();
  double2* dh = c->dh.as<double2>();
  double2* dh2 = c->dh2.as<double2>();
  double2* dn = c->dnrm.as<double2>();
  double2* dy = c->dy.as<double2>();
  int* flag = c->flag.as<int>();
  const RedScratch sc = scratch(c);
  const double sz = sizeof(C<T>);
  c->stream = c->cap[0];
  CK(cudaStreamBeginCapture(c->cap[0], cudaStreamCaptureModeThreadLocal));
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g0 = nullptr;
  CK(cudaStreamGetCaptureInfo(c->cap[0], &cs, nullptr, &g0, nullptr, nullptr, nullptr));
  // a handle serves one conditional node and belongs to the graph that holds it: the WHILE node sits
  // in the top graph, the m IF nodes (one handle each) in the WHILE body
  cudaGraphConditionalHandle h_outer;
  CK(cudaGraphConditionalHandleCreate(&h_outer, g0, 0, 0));
  c->tape = &G->pre;
  KL(IE_K_KRYLOV_MISC, sz * n, Krylov<T>::norm2(b, n, dn, sc, c->stream));
  KL(IE_K_KRYLOV_MISC, 0, gm_init(st, dn, h_outer, c->stream));
  CK(cudaMemsetAsync(x, 0, sizeof(C<T>) * n, c->stream));
  KL(IE_K_KRYLOV_MISC, 2 * sz * n, Krylov<T>::scale(b, V, n, dn, 0.0, c->stream));
  cudaGraph_t wbody = nullptr;
  CKS(add_conditional(c, c->cap[0], h_outer, cudaGraphCondTypeWhile, &wbody));
  GmSteps steps;
  steps.m = m;
  for (int j = 0; j < m; ++j) CK(cudaGraphConditionalHandleCreate(&steps.h[j], wbody, 0, 0));
  CK(cudaStreamBeginCaptureToGraph(c->cap[1], wbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  c->stream = c->cap[1];
  c->tape = &G->head;
  KL(IE_K_KRYLOV_MISC, 0, gm_cycle(st, steps, c->stream));
  G->step.assign(m, Tape());
  for (int j = 0; j < m; ++j) {
    cudaGraph_t ibody = nullptr;
    CKS(add_conditional(c, c->cap[1], steps.h[j], cudaGraphCondTypeIf, &ibody));
    CK(cudaStreamBeginCaptureToGraph(c->cap[2], ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    c->stream = c->cap[2];
    c->tape = &G->step[j];
    C<T>* w = V + (size_t)(j + 1) * ld;
    CKS(A.apply(V + (size_t)j * ld, w));
    const int nv = j + 1;
    const double ng = (nv + kDotGroup - 1) / kDotGroup;
    KL(IE_K_DOTS, sz * n * (nv + ng), Krylov<T>::dots(V, ld, nv, w, n, cgs2, dh, nullptr, nullptr, sc, c->stream));
    KL(IE_K_UPDATE, sz * n * (nv + 2),
       Krylov<T>::update(V, ld, nv, dh, w, n, dn, dh + nv, 0.5, cgs2 ? flag : nullptr, nullptr, sc, c->stream));
    if (cgs2) {
      KL(IE_K_DOTS, 0, Krylov<T>::dots(V, ld, nv, w, n, false, dh2, dh, flag, sc, c->stream));
      KL(IE_K_UPDATE, 0, Krylov<T>::update(V, ld, nv, dh2, w, n, dn, nullptr, 0.0, nullptr, flag, sc, c->stream));
    }
    KL(IE_K_KRYLOV_MISC, 2 * sz * n, Krylov<T>::scale(w, w, n, dn, 0.0, c->stream));
    KL(IE_K_KRYLOV_MISC, 0,
       gm_step(st, j, dh, dn, cgs2 ? flag : nullptr, steps.h[j + 1 < m ? j + 1 : j], j + 1 < m, c->stream));
    cudaGraph_t done = nullptr;
    CK(cudaStreamEndCapture(c->cap[2], &done));
    c->stream = c->cap[1];
  }
  c->tape = &G->tail;
  KL(IE_K_KRYLOV_MISC, 0, gm_solve(st, dy, c->stream));
  KL(IE_K_KRYLOV_MISC, 2 * sz * n, Krylov<T>::combine(V, ld, m, dy, x, n, c->stream, &st->jd));
  CKS(A.apply(x, tmp));
  KL(IE_K_KRYLOV_MISC, 3 * sz * n, Krylov<T>::rsub(b, tmp, n, dn + 1, sc, c->stream));
  KL(IE_K_KRYLOV_MISC, 0, gm_restart(st, dn + 1, h_outer, c->stream));
  KL(IE_K_KRYLOV_MISC, 2 * sz * n, Krylov<T>::scale(tmp, V, n, dn + 1, 0.0, c->stream));
  cudaGraph_t done1 = nullptr;
  CK(cudaStreamEndCapture(c->cap[1], &done1));
  c->stream = c->cap[0];
  CK(cudaStreamEndCapture(c->cap[0], &G->graph));
  CK(cudaGraphInstantiate(&G->exec, G->graph, 0));
  return IE_OK;
}

template <typename T> struct GraphRun {  // one launched GMRES graph whose results are still on the device
  GmGraph* G = nullptr;
  long n = 0;
  int m = 0;
};

// Launches GMRES as one CUDA graph on the context stream (see gmres_graph) without waiting for it:
// gmres_graph_finish reads its outcome. Several contexts' graphs can so run at the same time with one
// host synchronisation each at the end.
template <typename T>
ie_status gmres_graph_launch(ie_ctx* c, const BlockOp<T>& A, const C<T>* b, C<T>* x, double tol, int m, int max_it,
                             GraphRun<T>* run) {
  const bool cgs2 = tol < kReorthTol;
  const long n = 3 * A.nb();
  CKS(ensure_scalars(c));
  if (m < 1 || m > 127) return fail(c, IE_EINVAL, "restart must be in [1, 127]");
  const long ld = (n + 1) & ~1L;
  CK(c->V.ensure(sizeof(C<T>) * (size_t)(m + 1) * ld));
  CK(c->kt1.ensure(sizeof(C<T>) * (size_t)n));
  CK(c->gm_state.ensure(sizeof(GmState)));
  for (int k = 0; k < 3; ++k) CKS(cap_stream(c, k));
  C<T>* V = c->V.as<C<T>>();
  const bool f32 = std::is_same<T, float>::value;
  // the graph is keyed by everything its kernel arguments point at
  auto make_key = [&]() {
    return std::vector<const void*>{
        reinterpret_cast<const void*>(sizeof(C<T>)), reinterpret_cast<const void*>((long)A.z0),
        reinterpret_cast<const void*>((long)A.nz), reinterpret_cast<const void*>((long)A.contract),
        reinterpret_cast<const void*>((long)m), reinterpret_cast<const void*>((long)cgs2), b, x, V,
        reinterpret_cast<const void*>(ld), c->kt1.p, (f32 ? c->A32 : c->A64).p, (f32 ? c->B32 : c->B64).p,
        (f32 ? c->cw32 : c->cw64).p, A.S, c->gm_state.p, c->dh.p, c->part.p};
  };
  std::vector<const void*> key = make_key();
  GmGraph* G = nullptr;
  for (auto* g : c->gm_graphs)
    if (g->key == key) G = g;
  if (!G) {
    // outside any capture: allocates the block's workspaces and tunes its tiles before they are captured
    // (and may move the workspaces, so the key is taken again)
    CKS(A.apply(V, V + ld));
    key = make_key();
    for (auto* g : c->gm_graphs)
      if (g->key == key) G = g;
  }
  if (!G) {
    G = new (std::nothrow) GmGraph();
    if (!G) return fail(c, IE_ENOMEM, "graph cache");
    G->key = key;
    cudaStream_t saved = c->stream;
    Tape* saved_tape = c->tape;
    const ie_status bst = build_gmres_graph<T>(c, A, b, x, m, cgs2, n, ld, G);
    c->stream = saved;
    c->tape = saved_tape;
    if (bst != IE_OK) {
      abandon_capture(c);
      delete G;
      return bst;
    }
    if ((int)c->gm_graphs.size() >= kGmGraphCache) {
      delete c->gm_graphs.front();
      c->gm_graphs.erase(c->gm_graphs.begin());
    }
    c->gm_graphs.push_back(G);
  }
  GmState* st = c->gm_state.as<GmState>();
  cudaStream_t s = c->stream;
  // launch parameters: max_it, m, tol (contiguous in GmState)
  const size_t p0 = offsetof(GmHead, max_it), p1 = offsetof(GmHead, tol) + sizeof(double);
  unsigned char* stage = reinterpret_cast<unsigned char*>(c->hpin);
  GmHead hs;
  hs.max_it = max_it;
  hs.m = m;
  hs.tol = tol;
  std::memcpy(stage, reinterpret_cast<const unsigned char*>(&hs) + p0, p1 - p0);
  CK(cudaMemcpyAsync(reinterpret_cast<unsigned char*>(st) + p0, stage, p1 - p0, cudaMemcpyHostToDevice, s));
  CK(cudaGraphLaunch(G->exec, s));
  const size_t hdr = offsetof(GmState, cs), lens = 256;
  CK(cudaMemcpyAsync(stage, st, hdr, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(stage + lens, reinterpret_cast<unsigned char*>(st) + offsetof(GmState, cyc_len),
                     sizeof(int) * kGmMaxCycles, cudaMemcpyDeviceToHost, s));
  run->G = G;
  run->n = n;
  run->m = m;
  return IE_OK;
}

// Waits for a graph started by gmres_graph_launch and collects its outcome and launch accounting.
template <typename T> ie_status gmres_graph_finish(ie_ctx* c, const GraphRun<T>& run, GmresOut* out) {
  GmGraph* G = run.G;
  const long n = run.n;
  const int m = run.m;
  unsigned char* stage = reinterpret_cast<unsigned char*>(c->hpin);
  const size_t hdr = offsetof(GmState, cs), lens = 256;
  GmHead hs;
  *out = GmresOut();
  CK(sync(c));
  std::memcpy(&hs, stage, hdr);
  std::vector<int> cyc(kGmMaxCycles);
  std::memcpy(cyc.data(), stage + lens, sizeof(int) * kGmMaxCycles);
  // accounting of what ran: the setup once, per cycle its head, its steps and its tail
  account(c, G->pre);
  const int ncyc = std::min(hs.cycles, kGmMaxCycles);
  for (int k = 0; k < ncyc; ++k) {
    account(c, G->head);
    for (int j = 0; j < std::min(cyc[k], m); ++j) account(c, G->step[j]);
    account(c, G->tail);
    c->prof.bytes[IE_K_KRYLOV_MISC] += sizeof(C<T>) * (double)n * cyc[k];  // x += V y reads cyc[k] vectors
  }
  if (hs.reorth > 0 && hs.iters > 0) {  // second Gram-Schmidt passes at the mean basis size
    const double nv = std::max(1.0, (double)hs.iters / std::max(1, hs.cycles) / 2.0);
    c->prof.bytes[IE_K_DOTS] += hs.reorth * sizeof(C<T>) * (double)n * (nv + std::ceil(nv / kDotGroup));
    c->prof.bytes[IE_K_UPDATE] += hs.reorth * sizeof(C<T>) * (double)n * (nv + 2);
  }
  if (hs.status == 3) return fail(c, IE_ECUDA, "GMRES produced a non-finite residual");
  out->iters = hs.iters;
  out->matvecs = hs.iters + hs.cycles;
  out->reorth = hs.reorth;
  out->rel = hs.rel;
  out->converged = hs.status == 1;
  return IE_OK;
}

template <typename T>
ie_status gmres_graph(ie_ctx* c, const BlockOp<T>& A, const C<T>* b, C<T>* x, double tol, int m, int max_it,
                      GmresOut* out) {
  GraphRun<T> run;
  CKS(gmres_graph_launch<T>(c, A, b, x, tol, m, max_it, &run));
  return gmres_graph_finish<T>(c, run, out);
}

struct SolveCfg {
  int dd_mode;
  std::vector<int> split;
  int restart, max_outer, max_inner, precision, adaptive, contraction, graph;
  int outer_krylov, outer_restart, concurrent;
  double fixed_tol, tol, outer_inner_tol;
};

// Flexible GMRES on the whole-grid system (I - G dsigma) E = E0 (eq. 8) over the active sub-domains,
// right-preconditioned by one sweep of Algorithm 1 started from zero (Krylov outer iteration in place of
// the fixed-point sweeps, as the paper's conclusion proposes). The Arnoldi and preconditioned vectors are
// whole-grid fields with the slabs of inactive sub-domains zeroed, stored in VT: complex64 in mixed
// precision, with the operator applied by the complex64 convolution (its rounding, ~1e-7 of |z|, stays
// below the target), complex128 with the FP64-accurate double-float convolution in FP64 mode. In both
// the field E is complex128 and the true residual that starts every cycle and decides convergence is
// FP64-accurate. Classical Gram-Schmidt with the DGKS second pass and FP64 Givens rotations on the host.
// Each outer step costs one sweep, one whole-grid application and the orthogonalisation.
template <typename T, typename VT, class Sweep>
ie_status fgmres_outer(ie_ctx* c, const SolveCfg& cfg, const std::vector<char>& act, Sweep& sweep,
                       const std::function<ie_status(const float2*, float2*, double, int*)>& sweep64, double e0norm,
                       double* e, int* sweeps, ie_info* info, bool record, bool fast_ok) {
  constexpr bool f32 = std::is_same<VT, float>::value;
  using CV = C<VT>;
  const long N3 = 3 * c->N, nxy = (long)c->nx * c->ny;
  const long ld = (N3 + 1) & ~1L;  // even stride keeps every vector 16-byte aligned
  const int m = cfg.outer_restart;
  if (m < 1 || m > 127) return fail(c, IE_EINVAL, "outer restart must be in [1, 127]");
  cudaStream_t s = c->stream;
  CKS(ensure_scalars(c));
  SpecSet* S = nullptr;
  CKS(get_spec(c, c->nz, &S));
  CK(c->FV.ensure(sizeof(CV) * (size_t)(m + 1) * ld));
  CK(c->FZ.ensure(sizeof(CV) * (size_t)m * ld));
  CK(c->PR.ensure(sizeof(double2) * N3));
  CK(c->PZ.ensure(sizeof(double2) * N3));
  CV* V = c->FV.as<CV>();
  CV* Z = c->FZ.as<CV>();
  double2* PR = c->PR.as<double2>();
  double2* PZ = c->PZ.as<double2>();
  const RedScratch sc = scratch(c);
  double2* dh = c->dh.as<double2>();
  double2* dh2 = c->dh2.as<double2>();
  double2* dn = c->dnrm.as<double2>();
  int* flag = c->flag.as<int>();
  const double vb = sizeof(CV);
  auto mask = [&](auto* v) -> ie_status {  // zero the slabs of the sub-domains left out
    using E = std::remove_pointer_t<decltype(v)>;
    for (size_t i = 0; i + 1 < cfg.split.size(); ++i) {
      if (act[i]) continue;
      const long off = (long)cfg.split[i] * nxy, nb = (long)(cfg.split[i + 1] - cfg.split[i]) * nxy;
      for (int k = 0; k < 3; ++k) CK(cudaMemsetAsync(v + k * c->N + off, 0, sizeof(E) * nb, s));
    }
    return IE_OK;
  };
  // c128 field -> VT vector and back (plain copies in FP64 mode)
  auto to_vec = [&](const double2* src, CV* dst) -> ie_status {
    if constexpr (f32)
      KL(IE_K_FIELD, 24.0 * N3, launch_c128_to_c64(src, c->N, reinterpret_cast<float2*>(dst), c->N, c->N, s));
    else
      CK(cudaMemcpyAsync(dst, src, sizeof(double2) * N3, cudaMemcpyDeviceToDevice, s));
    return IE_OK;
  };
  auto to_field = [&](const CV* src, double2* dst) -> ie_status {  // dst := src
    if constexpr (f32) {
      CK(cudaMemsetAsync(dst, 0, sizeof(double2) * N3, s));
      KL(IE_K_FIELD, 40.0 * N3, launch_add_c64_to_c128(reinterpret_cast<const float2*>(src), c->N, dst, c->N, c->N, s));
    } else {
      CK(cudaMemcpyAsync(dst, src, sizeof(double2) * N3, cudaMemcpyDeviceToDevice, s));
    }
    return IE_OK;
  };
  std::vector<std::complex<double>> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  auto Hij = [&](int i, int j) -> std::complex<double>& { return H[(size_t)i * m + j]; };
  while (*e > cfg.tol && *sweeps < cfg.max_outer) {
    CKS(mask(c->R.as<double2>()));
    const double beta = *e * e0norm;  // |R| over the active slabs
    CKS(to_vec(c->R.as<double2>(), V));
    KL(IE_K_KRYLOV_MISC, 2.0 * vb * N3, Krylov<VT>::scale(V, V, N3, nullptr, 1.0 / beta, s));
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jd = 0;
    for (int j = 0; j < m && *sweeps < cfg.max_outer; ++j) {
      CV* vj = V + (size_t)j * ld;
      CV* zj = Z + (size_t)j * ld;
      CV* w = V + (size_t)(j + 1) * ld;
      int its = 0;
      if constexpr (f32) {
        if (sweep64) {  // z_j = M^-1 v_j straight between the complex64 outer vectors
          CKS(mask(zj));
          CKS(sweep64(reinterpret_cast<const float2*>(vj), reinterpret_cast<float2*>(zj), cfg.outer_inner_tol, &its));
        }
      }
      if (!(f32 && sweep64)) {
        CKS(to_field(vj, PR));
        CK(cudaMemsetAsync(PZ, 0, sizeof(double2) * N3, s));
        CKS(sweep(PR, PZ, cfg.outer_inner_tol, &its));
        CKS(to_vec(PZ, zj));
      }
      ++*sweeps;
      if constexpr (f32)
        CKS(conv<float>(c, S, zj, c->N, 0, c->nz, 0, c->nz, 0, EPI_APPLY, zj, c->N, w, c->N, nullptr, 0, nullptr, 0));
      else
        CKS(conv<df>(c, S, zj, c->N, 0, c->nz, 0, c->nz, 0, EPI_APPLY, zj, c->N, w, c->N, nullptr, 0, nullptr, 0));
      CKS(mask(w));
      const int nv = j + 1;
      const double ng = (nv + kDotGroup - 1) / kDotGroup;
      KL(IE_K_DOTS, vb * N3 * (nv + ng), Krylov<VT>::dots(V, ld, nv, w, N3, true, dh, nullptr, nullptr, sc, s));
      KL(IE_K_UPDATE, vb * N3 * (nv + 2),
         Krylov<VT>::update(V, ld, nv, dh, w, N3, dn, dh + nv, 0.5, flag, nullptr, sc, s));
      KL(IE_K_DOTS, 0, Krylov<VT>::dots(V, ld, nv, w, N3, false, dh2, dh, flag, sc, s));
      KL(IE_K_UPDATE, 0, Krylov<VT>::update(V, ld, nv, dh2, w, N3, dn, nullptr, 0.0, nullptr, flag, sc, s));
      KL(IE_K_KRYLOV_MISC, 2.0 * vb * N3, Krylov<VT>::scale(w, w, N3, dn, 0.0, s));
      CK(cudaMemcpyAsync(c->hpin, dh, sizeof(double2) * nv, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(c->hpin + nv, dn, sizeof(double2), cudaMemcpyDeviceToHost, s));
      CK(sync(c));
      for (int i = 0; i < nv; ++i) Hij(i, j) = std::complex<double>(c->hpin[i].x, c->hpin[i].y);
      const double hn = std::sqrt(std::max(c->hpin[nv].x, 0.0));
      Hij(j + 1, j) = hn;
      for (int i = 0; i < j; ++i) {
        const std::complex<double> t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -std::conj(sn[i]) * Hij(i, j) + std::conj(cs[i]) * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      const std::complex<double> a = Hij(j, j), d = Hij(j + 1, j);
      const double den = std::sqrt(std::norm(a) + std::norm(d));
      cs[j] = den != 0.0 ? std::conj(a) / den : 1.0;
      sn[j] = den != 0.0 ? std::conj(d) / den : 0.0;
      Hij(j, j) = cs[j] * a + sn[j] * d;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -std::conj(sn[j]) * g[j];
      g[j] = cs[j] * g[j];
      jd = j + 1;
      const double est = std::abs(g[j + 1]) / e0norm;
      if (!std::isfinite(est)) return fail(c, IE_ECUDA, "outer GMRES produced a non-finite residual");
      if (record && info->n_history < IE_MAX_HISTORY) {
        info->sweep_gmres_iters[info->n_history - 1] = its;
        info->residual_history[info->n_history++] = est;
      }
      if (est <= cfg.tol || hn == 0.0) break;
    }
    for (int i = jd - 1; i >= 0; --i) {  // back substitution
      std::complex<double> acc = g[i];
      for (int k = i + 1; k < jd; ++k) acc -= Hij(i, k) * y[k];
      y[i] = acc / Hij(i, i);
    }
    for (int i = 0; i < jd; ++i) c->hpin[i] = make_double2(y[i].real(), y[i].imag());
    CK(cudaMemcpyAsync(c->dy.as<double2>(), c->hpin, sizeof(double2) * jd, cudaMemcpyHostToDevice, s));
    if constexpr (f32) {  // E += Z y: the combination in complex64, added to the complex128 field
      CK(c->FW32.ensure(sizeof(float2) * N3));
      float2* zy = c->FW32.as<float2>();
      CK(cudaMemsetAsync(zy, 0, sizeof(float2) * N3, s));
      KL(IE_K_KRYLOV_MISC, vb * N3 * (jd + 2), Krylov<float>::combine(Z, ld, jd, c->dy.as<double2>(), zy, N3, s));
      KL(IE_K_FIELD, 40.0 * N3, launch_add_c64_to_c128(zy, c->N, c->E.as<double2>(), c->N, c->N, s));
    } else {
      KL(IE_K_KRYLOV_MISC, vb * N3 * (jd + 2),
         Krylov<double>::combine(Z, ld, jd, c->dy.as<double2>(), c->E.as<double2>(), N3, s));
    }
    CKS(full_residual(c, e0norm, e, fast_ok && *e > fast_residual_above(cfg.tol), fast_residual_above(cfg.tol)));
  }
  return IE_OK;
}

// Algorithm 1 (with FP64 refinement) for the source whose E0 is in c->E0; leaves E in c->E.
template <typename T>
ie_status solve_one(ie_ctx* c, const SolveCfg& cfg, ie_info* info, bool record) {
  cudaStream_t s = c->stream;
  const long nxy = (long)c->nx * c->ny;
  const int M = (int)cfg.split.size() - 1;
  const bool warm = c->has_init;
  c->has_init = false;  // an initial guess serves one source
  // Sub-domains without contrast are left out of the sweeps and e is measured over the anomalous
  // ones (Section 3.1); their field is filled in from the final residual (E + R = E0 + G dsigma E).
  std::vector<char> blk_active(M, 1);
  c->e_slabs.clear();
  if (cfg.dd_mode != IE_DD_NONE) {
    for (int i = 0; i < M; ++i) {
      char any = 0;
      for (int z = cfg.split[i]; z < cfg.split[i + 1]; ++z) any |= c->active[z];
      blk_active[i] = any;
      if (any) {
        if (!c->e_slabs.empty() && c->e_slabs.back().first + c->e_slabs.back().second == cfg.split[i])
          c->e_slabs.back().second += cfg.split[i + 1] - cfg.split[i];
        else
          c->e_slabs.emplace_back(cfg.split[i], cfg.split[i + 1] - cfg.split[i]);
      }
    }
    if (c->e_slabs.size() == 1 && c->e_slabs[0].first == 0 && c->e_slabs[0].second == c->nz) c->e_slabs.clear();
    info->active_blocks += (int)std::count(blk_active.begin(), blk_active.end(), 1);
    if (std::count(blk_active.begin(), blk_active.end(), 1) == 0) {  // no contrast anywhere: E = E0
      CK(cudaMemcpyAsync(c->E.p, c->E0.p, sizeof(double2) * 3 * c->N, cudaMemcpyDeviceToDevice, s));
      return IE_OK;
    }
  } else {
    info->active_blocks += 1;
  }
  CK(cudaMemcpyAsync(c->E.p, c->E0.p, sizeof(double2) * 3 * c->N, cudaMemcpyDeviceToDevice, s));
  double e0norm;
  CKS(slab_norm(c, c->E0.as<double2>(), &e0norm));
  if (e0norm == 0.0) return IE_OK;  // no incident field in the anomalous region: E = E0 there
  double e;
  const bool fast_ok = cfg.precision == IE_PREC_MIXED;  // complex128 mode keeps every residual in FP64
  CKS(full_residual(c, e0norm, &e, fast_ok, fast_residual_above(cfg.tol)));
  if (warm) {  // a given initial guess replaces E := E0 only if its residual is smaller
    const double e_cold = e;
    CK(cudaMemcpyAsync(c->E.p, c->Einit.p, sizeof(double2) * 3 * c->N, cudaMemcpyDeviceToDevice, s));
    CKS(full_residual(c, e0norm, &e, fast_ok, fast_residual_above(cfg.tol)));
    info->cold_rel_residual = e_cold;
    info->warm_rel_residual = e;
    if (e < e_cold) {
      info->warm_start_used = 1;
    } else {
      CK(cudaMemcpyAsync(c->E.p, c->E0.p, sizeof(double2) * 3 * c->N, cudaMemcpyDeviceToDevice, s));
      CKS(full_residual(c, e0norm, &e, fast_ok, fast_residual_above(cfg.tol)));
    }
  }
  if (record) {
    info->n_history = 1;
    info->residual_history[0] = e;
  }
  std::vector<BlockOp<T>> ops(M);
  long nbmax = 0;
  for (int i = 0; i < M; ++i) {
    CKS(make_block<T>(c, cfg.split[i], cfg.split[i + 1] - cfg.split[i], &ops[i], cfg.contraction != 0));
    nbmax = std::max(nbmax, ops[i].nb());
  }
  SpecSet* Sfull = nullptr;
  if (cfg.dd_mode == IE_DD_GAUSS_SEIDEL && M > 1) CKS(get_spec(c, c->nz, &Sfull));
  CK(c->kb.ensure(sizeof(C<T>) * 3 * nbmax));
  CK(c->kx.ensure(sizeof(C<T>) * 3 * nbmax));
  CK(c->kt2.ensure(sizeof(C<T>) * 3 * nbmax));
  C<T>* rhs = c->kb.as<C<T>>();
  C<T>* dx = c->kx.as<C<T>>();
  C<T>* t2 = c->kt2.as<C<T>>();
  // complex64 DD solves keep A_ii E_i of every block: formed once here, then advanced by A_ii delta =
  // rhs - (final GMRES residual) after each block solve, so |b_i| = |R_i + A_ii E_i| costs a norm
  // instead of an operator application per block and sweep
  const bool keep_ae = std::is_same<T, float>::value && cfg.dd_mode != IE_DD_NONE;
  std::vector<long> ae_off(M, 0);
  if (keep_ae) {
    long tot = 0;
    for (int i = 0; i < M; ++i) {
      ae_off[i] = tot;
      tot += 3 * ops[i].nb();
    }
    CK(c->AEb.ensure(sizeof(float2) * tot));
    for (int i = 0; i < M; ++i) {
      if (!blk_active[i]) continue;
      const long nb = ops[i].nb(), off = (long)ops[i].z0 * nxy;
      KL(IE_K_FIELD, 72.0 * nb,
         launch_c128_to_c64(c->E.as<double2>() + off, c->N, reinterpret_cast<float2*>(dx), nb, nb, s));
      CKS(ops[i].apply_conv(dx, reinterpret_cast<C<T>*>(c->AEb.as<float2>() + ae_off[i])));
    }
  }
  // One sweep of Algorithm 1 over the active blocks on the residual Rb, accumulating the corrections into
  // Eb. precond_tol <= 0: the sweep of the fixed-point iteration (block tolerance e/10 relative to
  // |b_i| = |R_i + A_ii E_i|). precond_tol > 0: a preconditioner application started from Eb = 0, so
  // b_i = R_i and every block is solved to precond_tol.
  bool inner_ok = true;
  auto sweep = [&](double2* Rb, double2* Eb, double precond_tol, int* sweep_its) -> ie_status {
    const bool pre = precond_tol > 0;
    for (int i = 0; i < M; ++i) {
      if (!blk_active[i]) continue;
      const BlockOp<T>& A = ops[i];
      const long nb = A.nb(), off = (long)A.z0 * nxy;
      double2* Ri = Rb + off;
      double2* Ei = Eb + off;
      double rnorm;
      CKS(norm_c128(c, Ri, c->N, nullptr, 0, nb, &rnorm));
      if (rnorm == 0.0) continue;
      // block right-hand side norm |b_i| = |R_i + A_ii E_i| (eqs. 21/23)
      double bnorm = rnorm;
      if (pre) {
      } else if (cfg.dd_mode == IE_DD_NONE) {
        CKS(norm_c128(c, c->E0.as<double2>(), c->N, nullptr, 0, c->N, &bnorm));
      } else if (keep_ae) {
        CKS(norm_c128(c, Ri, c->N, c->AEb.as<float2>() + ae_off[i], nb, nb, &bnorm));
      } else if (std::is_same<T, float>::value) {
        KL(IE_K_FIELD, 72.0 * nb, launch_c128_to_c64(Ei, c->N, reinterpret_cast<float2*>(dx), nb, nb, s));
        CKS(A.apply_conv(dx, t2));
        CKS(norm_c128(c, Ri, c->N, reinterpret_cast<const float2*>(t2), nb, nb, &bnorm));
      } else {
        KL(IE_K_FIELD, 96.0 * nb, launch_copy_c128(Ei, c->N, reinterpret_cast<double2*>(dx), nb, nb, s));
        CKS(A.apply_conv(dx, t2));
        KL(IE_K_FIELD, 144.0 * nb, launch_add_c128(Ri, c->N, reinterpret_cast<double2*>(t2), nb, nb, s));
        CKS(norm_c128(c, reinterpret_cast<const double2*>(t2), nb, nullptr, 0, nb, &bnorm));
      }
      double tol_i;
      if (pre) {
        tol_i = precond_tol;
      } else {
        const double target = (cfg.dd_mode == IE_DD_NONE) ? cfg.tol : (cfg.adaptive ? e / 10.0 : cfg.fixed_tol);
        tol_i = target * bnorm / rnorm;
      }
      if (std::is_same<T, float>::value) tol_i = std::max(tol_i, cfg.dd_mode == IE_DD_NONE ? 1e-5 : 1e-6);
      tol_i = std::min(tol_i, 0.5);
      if (std::is_same<T, float>::value)
        KL(IE_K_FIELD, 72.0 * nb, launch_c128_to_c64(Ri, c->N, reinterpret_cast<float2*>(rhs), nb, nb, s));
      else
        KL(IE_K_FIELD, 96.0 * nb, launch_copy_c128(Ri, c->N, reinterpret_cast<double2*>(rhs), nb, nb, s));
      GmresOut go;
      if (cfg.graph)
        CKS(gmres_graph<T>(c, A, rhs, dx, tol_i, cfg.restart, cfg.max_inner, &go));
      else
        CKS(gmres<T>(c, A, rhs, dx, true, tol_i, cfg.restart, cfg.max_inner, &go, !pre));
      if (keep_ae && !pre && go.iters > 0)  // A_ii delta = rhs - r, r = rhs - A x the final true residual
        KL(IE_K_FIELD, 96.0 * nb,
           launch_add_diff_c64(c->AEb.as<float2>() + ae_off[i], reinterpret_cast<const float2*>(rhs),
                               c->kt1.as<float2>(), 3 * nb, s));
      CKS(A.to_field(dx));  // contraction form: the field correction is M times the GMRES solution
      inner_ok = inner_ok && go.converged;
      *sweep_its += go.iters;
      info->gmres_iters_total += go.iters;
      info->reorth_passes += go.reorth;
      info->matvecs += go.matvecs;
      if (std::is_same<T, float>::value)
        KL(IE_K_FIELD, 120.0 * nb, launch_add_c64_to_c128(reinterpret_cast<const float2*>(dx), nb, Ei, c->N, nb, s));
      else
        KL(IE_K_FIELD, 144.0 * nb, launch_add_c128(reinterpret_cast<const double2*>(dx), nb, Ei, c->N, nb, s));
      if (cfg.dd_mode == IE_DD_GAUSS_SEIDEL) {
        for (int j = i + 1; j < M; ++j) {  // interaction update of the later blocks (eq. 21)
          if (!blk_active[j]) continue;
          const BlockOp<T>& Bj = ops[j];
          CKS(conv<T>(c, Sfull, dx, nb, A.z0, A.nz, A.z0, Bj.nz, Bj.z0, EPI_ACCUM128, nullptr, 0, nullptr, 0,
                      Rb + (long)Bj.z0 * nxy, c->N, nullptr, 0));
        }
      }
    }
    return IE_OK;
  };
  // The same sweep for block Jacobi with the sub-domain solves in flight together (concurrent_blocks):
  // norms, tolerances and right-hand sides are formed on the context stream as above, then every block
  // is solved by its worker context (own stream, own Krylov basis) on its own host thread, and the
  // corrections are added to the whole-grid field on the context stream. Eq. 23: in a Jacobi sweep the
  // block solves read only the previous sweep's field, so they are independent.
  const bool conc = cfg.concurrent && cfg.dd_mode == IE_DD_JACOBI && M > 1;
  if (conc) CKS(prepare_workers(c, cfg.split));
  // v64/z64 (complex64 preconditioner application of the outer Krylov iteration, z = M^-1 v with the
  // whole-grid layout of the outer basis): each block's right-hand side is copied from v64's slab and its
  // solution to z64's slab, with no complex128 field in between; Rb and Eb are then unused.
  auto sweep_conc_io = [&](double2* Rb, double2* Eb, const float2* v64, float2* z64, double precond_tol,
                           int* sweep_its) -> ie_status {
    const bool pre = precond_tol > 0;
    const bool direct = v64 != nullptr && std::is_same<T, float>::value;
    struct Job {
      int i = 0;
      double tol = 0.0;
      GmresOut go;
      ie_status st = IE_OK;
    };
    std::vector<Job> jobs;
    for (int i = 0; i < M; ++i) {
      if (!blk_active[i]) continue;
      const BlockOp<T>& A = ops[i];
      const long nb = A.nb(), off = (long)A.z0 * nxy;
      ie_ctx* w = c->workers[i];
      if (direct) {  // a zero right-hand side gives a zero solution inside the block solve
        CK(w->kb.ensure(sizeof(C<T>) * 3 * nb));
        CK(w->kx.ensure(sizeof(C<T>) * 3 * nb));
        CK(cudaMemcpy2DAsync(w->kb.p, sizeof(float2) * nb, v64 + off, sizeof(float2) * c->N, sizeof(float2) * nb, 3,
                             cudaMemcpyDeviceToDevice, s));
        Job j;
        j.i = i;
        j.tol = std::min(std::max(precond_tol, 1e-6), 0.5);
        jobs.push_back(j);
        continue;
      }
      double2* Ri = Rb + off;
      double2* Ei = Eb + off;
      double rnorm;
      CKS(norm_c128(c, Ri, c->N, nullptr, 0, nb, &rnorm));
      if (rnorm == 0.0) continue;
      double bnorm = rnorm;  // |b_i| = |R_i + A_ii E_i| (eq. 23)
      if (pre) {
      } else if (keep_ae) {
        CKS(norm_c128(c, Ri, c->N, c->AEb.as<float2>() + ae_off[i], nb, nb, &bnorm));
      } else if (std::is_same<T, float>::value) {
        KL(IE_K_FIELD, 72.0 * nb, launch_c128_to_c64(Ei, c->N, reinterpret_cast<float2*>(dx), nb, nb, s));
        CKS(A.apply_conv(dx, t2));
        CKS(norm_c128(c, Ri, c->N, reinterpret_cast<const float2*>(t2), nb, nb, &bnorm));
      } else {
        KL(IE_K_FIELD, 96.0 * nb, launch_copy_c128(Ei, c->N, reinterpret_cast<double2*>(dx), nb, nb, s));
        CKS(A.apply_conv(dx, t2));
        KL(IE_K_FIELD, 144.0 * nb, launch_add_c128(Ri, c->N, reinterpret_cast<double2*>(t2), nb, nb, s));
        CKS(norm_c128(c, reinterpret_cast<const double2*>(t2), nb, nullptr, 0, nb, &bnorm));
      }
      double tol_i = pre ? precond_tol : (cfg.adaptive ? e / 10.0 : cfg.fixed_tol) * bnorm / rnorm;
      if (std::is_same<T, float>::value) tol_i = std::max(tol_i, 1e-6);
      tol_i = std::min(tol_i, 0.5);
      CK(w->kb.ensure(sizeof(C<T>) * 3 * nb));
      CK(w->kx.ensure(sizeof(C<T>) * 3 * nb));
      if (std::is_same<T, float>::value)
        KL(IE_K_FIELD, 72.0 * nb, launch_c128_to_c64(Ri, c->N, w->kb.as<float2>(), nb, nb, s));
      else
        KL(IE_K_FIELD, 96.0 * nb, launch_copy_c128(Ri, c->N, w->kb.as<double2>(), nb, nb, s));
      Job j;
      j.i = i;
      j.tol = tol_i;
      jobs.push_back(j);
    }
    if (jobs.empty()) return IE_OK;
    cudaEvent_t ev = nullptr;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    const ie_status ost = order_workers(c, ev);
    cudaEventDestroy(ev);  // released once the recorded work completes
    CKS(ost);
    if (cfg.graph) {
      // device-driven block solves: each block's GMRES graph is launched on its worker stream from this
      // thread, all of them before the first wait, so the whole sweep runs on the GPU with one host
      // synchronisation per block at its end
      std::vector<GraphRun<T>> runs(jobs.size());
      std::vector<BlockOp<T>> wops(jobs.size());
      for (size_t k = 0; k < jobs.size(); ++k) {
        ie_ctx* w = c->workers[jobs[k].i];
        jobs[k].st = make_block<T>(w, 0, w->nz, &wops[k], cfg.contraction != 0);
        if (jobs[k].st == IE_OK)
          jobs[k].st = gmres_graph_launch<T>(w, wops[k], w->kb.template as<C<T>>(), w->kx.template as<C<T>>(),
                                             jobs[k].tol, cfg.restart, cfg.max_inner, &runs[k]);
      }
      for (size_t k = 0; k < jobs.size(); ++k) {
        ie_ctx* w = c->workers[jobs[k].i];
        if (jobs[k].st == IE_OK) jobs[k].st = gmres_graph_finish<T>(w, runs[k], &jobs[k].go);
        if (jobs[k].st == IE_OK) jobs[k].st = wops[k].to_field(w->kx.template as<C<T>>());
      }
      for (size_t k = 0; k < jobs.size(); ++k) {
        ie_ctx* w = c->workers[jobs[k].i];
        if (sync(w) != cudaSuccess && jobs[k].st == IE_OK) jobs[k].st = fail(w, IE_ECUDA, "sub-domain solve on its stream");
      }
    }
    std::vector<std::thread> pool;  // host-driven block solves: one host thread per block
    for (auto& job : jobs) {
      if (cfg.graph) break;
      pool.emplace_back([&, jp = &job]() {
        cudaSetDevice(c->dev);
        ie_ctx* w = c->workers[jp->i];
        BlockOp<T> A;
        jp->st = make_block<T>(w, 0, w->nz, &A, cfg.contraction != 0);
        C<T>* rhs_w = w->kb.template as<C<T>>();
        C<T>* dx_w = w->kx.template as<C<T>>();
        if (jp->st == IE_OK)
          jp->st = gmres<T>(w, A, rhs_w, dx_w, true, jp->tol, cfg.restart, cfg.max_inner, &jp->go, !pre);
        if (jp->st == IE_OK) jp->st = A.to_field(dx_w);
        if (jp->st == IE_OK && sync(w) != cudaSuccess) jp->st = fail(w, IE_ECUDA, "sub-domain solve on its stream");
      });
    }
    for (auto& t : pool) t.join();
    for (const auto& job : jobs)
      if (job.st != IE_OK) return fail(c, job.st, "sub-domain " + std::to_string(job.i) + ": " + c->workers[job.i]->err);
    for (const auto& job : jobs) {  // every worker stream has drained: add the corrections
      ie_ctx* w = c->workers[job.i];
      fold_profile(c, w);
      const long nb = ops[job.i].nb(), off = (long)ops[job.i].z0 * nxy;
      if (direct) {
        CK(cudaMemcpy2DAsync(z64 + off, sizeof(float2) * c->N, w->kx.p, sizeof(float2) * nb, sizeof(float2) * nb, 3,
                             cudaMemcpyDeviceToDevice, s));
      } else {
        double2* Ei = Eb + off;
        if (keep_ae && !pre && job.go.iters > 0)  // A_ii delta = rhs - r (r: the final true residual)
          KL(IE_K_FIELD, 96.0 * nb,
             launch_add_diff_c64(c->AEb.as<float2>() + ae_off[job.i], w->kb.as<float2>(), w->kt1.as<float2>(),
                                 3 * nb, s));
        if (std::is_same<T, float>::value)
          KL(IE_K_FIELD, 120.0 * nb, launch_add_c64_to_c128(w->kx.as<float2>(), nb, Ei, c->N, nb, s));
        else
          KL(IE_K_FIELD, 144.0 * nb, launch_add_c128(w->kx.as<double2>(), nb, Ei, c->N, nb, s));
      }
      inner_ok = inner_ok && job.go.converged;
      *sweep_its += job.go.iters;
      info->gmres_iters_total += job.go.iters;
      info->reorth_passes += job.go.reorth;
      info->matvecs += job.go.matvecs;
    }
    return IE_OK;
  };
  auto sweep_conc = [&](double2* Rb, double2* Eb, double precond_tol, int* sweep_its) -> ie_status {
    return sweep_conc_io(Rb, Eb, nullptr, nullptr, precond_tol, sweep_its);
  };
  auto sweep_any = [&](double2* Rb, double2* Eb, double precond_tol, int* sweep_its) -> ie_status {
    return conc ? sweep_conc(Rb, Eb, precond_tol, sweep_its) : sweep(Rb, Eb, precond_tol, sweep_its);
  };
  // complex64 preconditioner for the outer iteration (concurrent block Jacobi in complex64 only)
  std::function<ie_status(const float2*, float2*, double, int*)> sweep64;
  if (conc && std::is_same<T, float>::value)
    sweep64 = [&](const float2* v, float2* z, double tol, int* its) -> ie_status {
      return sweep_conc_io(nullptr, nullptr, v, z, tol, its);
    };
  int sweeps = 0;
  if (cfg.outer_krylov && cfg.dd_mode != IE_DD_NONE) {
    const ie_status ost =
        fast_ok ? fgmres_outer<T, float>(c, cfg, blk_active, sweep_any, sweep64, e0norm, &e, &sweeps, info, record,
                                         fast_ok)
                : fgmres_outer<T, double>(c, cfg, blk_active, sweep_any, sweep64, e0norm, &e, &sweeps, info, record,
                                          fast_ok);
    CKS(ost);
  } else {
    while (e > cfg.tol && sweeps < cfg.max_outer) {
      int sweep_its = 0;
      CKS(sweep_any(c->R.as<double2>(), c->E.as<double2>(), 0.0, &sweep_its));
      sweeps++;
      CKS(full_residual(c, e0norm, &e, fast_ok && e > fast_residual_above(cfg.tol), fast_residual_above(cfg.tol)));
      if (record && info->n_history < IE_MAX_HISTORY) {
        info->sweep_gmres_iters[info->n_history - 1] = sweep_its;
        info->residual_history[info->n_history++] = e;
      }
    }
  }
  info->outer_iters += sweeps;
  info->final_rel_residual = std::max(info->final_rel_residual, e);
  for (int i = 0; i < M; ++i) {  // field of the sub-domains left out: E0 + G dsigma E = E + R
    if (blk_active[i]) continue;
    const long nb = ops[i].nb(), off = (long)ops[i].z0 * nxy;
    KL(IE_K_FIELD, 144.0 * nb, launch_add_c128(c->R.as<double2>() + off, c->N, c->E.as<double2>() + off, c->N, nb, s));
  }
  if (e > cfg.tol) return IE_ENOCONV;
  return IE_OK;
}

ie_status upload_c128(ie_ctx* c, const double* host, long n, DevBuf& dst) {
  CK(dst.ensure(sizeof(double2) * n));
  CK(cudaMemcpyAsync(dst.p, host, sizeof(double2) * n, cudaMemcpyHostToDevice, c->stream));
  return IE_OK;
}

}  // namespace

template <typename T>
ie_status gmres_host(ie_ctx* c, int z0, int nz, const double* b, const double* x0, double tol, int restart,
                            int max_iter, double* x, int32_t* iters, double* rel) {
  BlockOp<T> A;
  CKS(make_block<T>(c, z0, nz, &A));
  const long n = 3 * A.nb();
  DevBuf bd, xd, bs, xs;
  CKS(upload_c128(c, b, n, bd));
  if (x0) CKS(upload_c128(c, x0, n, xd));
  else CK(xd.ensure(sizeof(double2) * n));
  C<T>* bb;
  C<T>* xx;
  if (std::is_same<T, float>::value) {
    CK(bs.ensure(sizeof(float2) * n));
    CK(xs.ensure(sizeof(float2) * n));
    const long nb = A.nb();
    KL(IE_K_FIELD, 72.0 * nb, launch_c128_to_c64(bd.as<double2>(), nb, bs.as<float2>(), nb, nb, c->stream));
    bb = bs.as<C<T>>();
    xx = xs.as<C<T>>();
    if (x0) KL(IE_K_FIELD, 72.0 * nb, launch_c128_to_c64(xd.as<double2>(), nb, xs.as<float2>(), nb, nb, c->stream));
  } else {
    bb = bd.as<C<T>>();
    xx = xd.as<C<T>>();
  }
  GmresOut go;
  CKS(gmres<T>(c, A, bb, xx, x0 == nullptr, tol, restart, max_iter, &go));
  if (std::is_same<T, float>::value) {
    CK(cudaMemsetAsync(xd.p, 0, sizeof(double2) * n, c->stream));
    KL(IE_K_FIELD, 120.0 * A.nb(), launch_add_c64_to_c128(xs.as<float2>(), A.nb(), xd.as<double2>(), A.nb(), A.nb(), c->stream));
  }
  CK(cudaMemcpyAsync(x, xd.p, sizeof(double2) * n, cudaMemcpyDeviceToHost, c->stream));
  CK(sync(c));
  if (iters) *iters = go.iters;
  if (rel) *rel = go.rel;
  return go.converged ? IE_OK : IE_ENOCONV;
}

// =============================================================================== C ABI
extern "C" {

void ie_default_opts(ie_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->n_blocks = 1;
  o->z_split = nullptr;
  o->restart = 30;
  o->max_outer = 50;
  o->max_inner = 600;
  o->precision = IE_PREC_MIXED;
  o->adaptive = 1;
  o->fixed_tol = 1e-6;
}

ie_status ie_create(const ie_grid* grid, double h, double sigma0, double freq, ie_ctx** out) {
  if (!out) return IE_EINVAL;
  *out = nullptr;
  if (!grid || !(h > 0) || !(sigma0 > 0) || !(freq > 0) || !std::isfinite(h) || !std::isfinite(sigma0) ||
      !std::isfinite(freq))
    return IE_EINVAL;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || grid->nx > 512 || grid->ny > 512 || grid->nz > 512)
    return IE_EINVAL;
  auto* c = new (std::nothrow) ie_ctx();
  if (!c) return IE_ENOMEM;
  if (cudaGetDevice(&c->dev) != cudaSuccess) {
    delete c;
    return IE_ECUDA;
  }
  c->nx = grid->nx;
  c->ny = grid->ny;
  c->nz = grid->nz;
  c->N = (long)c->nx * c->ny * c->nz;
  for (int a = 0; a < 3; ++a) c->origin[a] = grid->origin[a];
  c->h = h;
  c->sigma0 = sigma0;
  c->freq = freq;
  c->omega = 2.0 * M_PI * freq;
  const std::complex<double> k = std::sqrt(std::complex<double>(0.0, c->omega * kMu0 * sigma0));
  c->k0 = make_double2(k.real(), k.imag());
  const double dv = h * h * h, a = std::cbrt(3.0 * dv / (4.0 * M_PI));
  const std::complex<double> ika(0.0, 1.0);
  const std::complex<double> self =
      ((2.0 / 3.0) * (1.0 - ika * k * a) * std::exp(ika * k * a) - 1.0) / sigma0;  // Section 2.2 self term
  c->self = make_double2(self.real(), self.imag());
  c->Lx = next_pow2(2 * c->nx);
  c->Ly = next_pow2(2 * c->ny);
  if (!supported_pencil(c->Lx) || !supported_pencil(c->Ly)) {
    delete c;
    return IE_EINVAL;
  }
  if (cudaHostAlloc(reinterpret_cast<void**>(&c->kerr), sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
    c->kerr = nullptr;
    delete c;
    return IE_ENOMEM;
  }
  *c->kerr = 0;
  // twiddles exp(-2 pi i k / TWN) in FP64 (angles reduced to the first octant by symmetry)
  std::vector<double2> t64(TWN);
  std::vector<float2> t32(TWN);
  std::vector<dfc> tdf(TWN);
  for (int q = 0; q < TWN; ++q) {
    const double ang = 2.0 * M_PI * (double)q / TWN;
    const double cr = std::cos(ang), si = std::sin(ang);
    t64[q] = make_double2(cr, -si);
    t32[q] = make_float2((float)cr, (float)-si);
    tdf[q] = dfc{df(cr), df(-si)};
  }
  if (c->tw64.ensure(sizeof(double2) * TWN) != cudaSuccess || c->tw32.ensure(sizeof(float2) * TWN) != cudaSuccess ||
      c->twdf.ensure(sizeof(dfc) * TWN) != cudaSuccess ||
      cudaMemcpy(c->tw64.p, t64.data(), sizeof(double2) * TWN, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->tw32.p, t32.data(), sizeof(float2) * TWN, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->twdf.p, tdf.data(), sizeof(dfc) * TWN, cudaMemcpyHostToDevice) != cudaSuccess ||
      c->E.ensure(sizeof(double2) * 3 * c->N) != cudaSuccess || c->E0.ensure(sizeof(double2) * 3 * c->N) != cudaSuccess ||
      c->R.ensure(sizeof(double2) * 3 * c->N) != cudaSuccess || c->ds64.ensure(sizeof(double) * 6 * c->N) != cudaSuccess ||
      c->ds32.ensure(sizeof(float) * 6 * c->N) != cudaSuccess) {
    delete c;
    return IE_ENOMEM;
  }
  SpecSet* S = nullptr;
  if (get_spec(c, c->nz, &S) != IE_OK) {  // whole-grid spectra (FP64 residual, interactions)
    const ie_status st = c->err.find("alloc") != std::string::npos ? IE_ENOMEM : IE_ECUDA;
    delete c;
    return st;
  }
  *out = c;
  return IE_OK;
}

ie_status ie_set_stream(ie_ctx* c, void* stream) {
  IE_ON_CTX_DEVICE(c);
  if (!c) return IE_EINVAL;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  return IE_OK;
}

static ie_status set_contrast_dev_impl(ie_ctx* c, const double* s6_dev) {
  CKS(ensure_scalars(c));
  int* flag = c->flag.as<int>();
  CK(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  KL(IE_K_FIELD, 120.0 * c->N,
     launch_set_contrast(s6_dev, c->N, c->sigma0, c->ds64.as<double>(), c->ds32.as<float>(), flag, c->stream));
  int bad = 0;
  CK(cudaMemcpyAsync(&c->hpin[0], flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(sync(c));
  std::memcpy(&bad, &c->hpin[0], sizeof(int));
  if (bad) {
    c->has_contrast = false;
    return fail(c, IE_EINVAL, "conductivity not finite or not positive definite");
  }
  // planes with contrast (sub-domains without any are left out of the DD sweeps)
  CK(c->plane_act.ensure(sizeof(int) * c->nz));
  KL(IE_K_FIELD, 48.0 * c->N,
     launch_plane_active(c->ds64.as<double>(), c->N, (long)c->nx * c->ny, c->nz, c->plane_act.as<int>(), c->stream));
  std::vector<int> act(c->nz);
  CK(cudaMemcpyAsync(act.data(), c->plane_act.p, sizeof(int) * c->nz, cudaMemcpyDeviceToHost, c->stream));
  CK(sync(c));
  c->active.assign(act.begin(), act.end());
  c->has_contrast = true;
  c->has_field = false;
  c->contract_ready = false;
  c->contrast_version++;
  return IE_OK;
}

ie_status ie_set_contrast(ie_ctx* c, const double* sigma6) {
  IE_ON_CTX_DEVICE(c);
  if (!c || !sigma6) return fail(c, IE_EINVAL, "null argument");
  CK(c->s6_stage.ensure(sizeof(double) * 6 * c->N));
  CK(cudaMemcpyAsync(c->s6_stage.p, sigma6, sizeof(double) * 6 * c->N, cudaMemcpyHostToDevice, c->stream));
  return set_contrast_dev_impl(c, c->s6_stage.as<double>());
}

ie_status ie_set_contrast_dev(ie_ctx* c, const double* sigma6_dev) {
  IE_ON_CTX_DEVICE(c);
  if (!c || !sigma6_dev) return fail(c, IE_EINVAL, "null argument");
  return set_contrast_dev_impl(c, sigma6_dev);
}

ie_status ie_solve(ie_ctx* c, int32_t n_src, const ie_dipole* src, int32_t n_rx, const double* rx, int32_t dd_mode,
                   double tol, const ie_opts* opts, double* H_out, ie_info* info) {
  IE_ON_CTX_DEVICE(c);
  const auto t0 = std::chrono::steady_clock::now();
  if (!c) return IE_EINVAL;
  c->err.clear();
  if (n_src < 0 || n_rx < 0 || (n_src > 0 && !src) || (n_rx > 0 && (!rx || !H_out)) || !(tol > 0))
    return fail(c, IE_EINVAL, "bad arguments");
  if (dd_mode != IE_DD_NONE && dd_mode != IE_DD_JACOBI && dd_mode != IE_DD_GAUSS_SEIDEL)
    return fail(c, IE_EINVAL, "bad dd_mode");
  if (!c->has_contrast) return fail(c, IE_ESTATE, "ie_set_contrast has not succeeded");
  ie_opts o;
  ie_default_opts(&o);
  if (opts) o = *opts;
  SolveCfg cfg;
  cfg.dd_mode = dd_mode;
  cfg.restart = o.restart > 0 ? o.restart : 30;
  cfg.max_outer = o.max_outer > 0 ? o.max_outer : 50;
  cfg.max_inner = o.max_inner > 0 ? o.max_inner : 20 * cfg.restart;
  cfg.precision = o.precision;
  cfg.adaptive = o.adaptive;
  cfg.fixed_tol = o.fixed_tol > 0 ? o.fixed_tol : tol;
  cfg.tol = tol;
  cfg.contraction = o.contraction;
  cfg.graph = o.graph;
  cfg.outer_krylov = o.outer_krylov;
  cfg.outer_restart = o.outer_restart > 0 ? o.outer_restart : 10;
  cfg.outer_inner_tol = o.outer_inner_tol > 0 ? o.outer_inner_tol : 0.1;
  cfg.concurrent = o.concurrent_blocks;
  if (o.concurrent_blocks != 0 && o.concurrent_blocks != 1) return fail(c, IE_EINVAL, "concurrent_blocks must be 0 or 1");
  if (o.outer_krylov != 0 && o.outer_krylov != 1) return fail(c, IE_EINVAL, "outer_krylov must be 0 or 1");
  if (o.graph != 0 && o.graph != 1) return fail(c, IE_EINVAL, "graph must be 0 or 1");
  if (o.contraction != 0 && o.contraction != 1) return fail(c, IE_EINVAL, "contraction must be 0 or 1");
  if (cfg.precision != IE_PREC_MIXED && cfg.precision != IE_PREC_FP64) return fail(c, IE_EINVAL, "bad precision");
  const int M = (dd_mode == IE_DD_NONE) ? 1 : std::max(1, o.n_blocks);
  if (M > c->nz) return fail(c, IE_EINVAL, "more blocks than z cells");
  cfg.split.resize(M + 1);
  if (dd_mode != IE_DD_NONE && o.z_split) {
    for (int i = 0; i <= M; ++i) cfg.split[i] = o.z_split[i];
    if (cfg.split[0] != 0 || cfg.split[M] != c->nz) return fail(c, IE_EINVAL, "z_split must run from 0 to nz");
    for (int i = 0; i < M; ++i)
      if (cfg.split[i + 1] <= cfg.split[i]) return fail(c, IE_EINVAL, "z_split must increase");
  } else {
    for (int i = 0; i <= M; ++i) cfg.split[i] = (int)((long)c->nz * i / M);
  }
  for (int q = 0; q < n_src; ++q) CKS(check_point(c, src[q].pos));
  for (int r = 0; r < n_rx; ++r) CKS(check_point(c, rx + 3 * r));
  ie_info loc;
  std::memset(&loc, 0, sizeof(loc));
  CKS(ensure_scalars(c));
  if (n_rx > 0) {
    CK(c->rxdev.ensure(sizeof(double) * 3 * n_rx));
    CK(c->Hdev.ensure(sizeof(double2) * 3 * n_rx));
    CK(c->rxpart.ensure(sizeof(double2) * 3 * kMaxRx * receivers_partials_blocks(c->N)));
    CK(cudaMemcpyAsync(c->rxdev.p, rx, sizeof(double) * 3 * n_rx, cudaMemcpyHostToDevice, c->stream));
  }
  ie_status worst = IE_OK;
  for (int q = 0; q < n_src; ++q) {
    KL(IE_K_FIELD, 48.0 * c->N,
       launch_incident_E(c->E0.as<double2>(), c->nx, c->ny, c->nz, c->origin, c->h, src[q].pos, src[q].moment, c->k0,
                         c->omega * kMu0, c->stream));
    ie_status st = cfg.precision == IE_PREC_FP64 ? solve_one<double>(c, cfg, &loc, q == 0)
                                                 : solve_one<float>(c, cfg, &loc, q == 0);
    if (st != IE_OK && st != IE_ENOCONV) return st;
    if (st == IE_ENOCONV) worst = IE_ENOCONV;
    c->has_field = true;
    for (int r0 = 0; r0 < n_rx; r0 += kMaxRx) {
      const int nr = std::min(kMaxRx, n_rx - r0);
      KL(IE_K_FIELD, 96.0 * c->N,
         launch_receivers(c->E.as<double2>(), c->N, c->ds64.as<double>(), c->N, c->nx, c->ny, c->origin, c->h,
                          c->rxdev.as<double>() + 3 * r0, nr, c->k0, c->rxpart.as<double2>(), src[q].pos,
                          src[q].moment, c->Hdev.as<double2>() + 3 * r0, c->stream));
    }
    if (n_rx > 0) {
      CK(cudaMemcpyAsync(H_out + (size_t)q * n_rx * 6, c->Hdev.p, sizeof(double2) * 3 * n_rx, cudaMemcpyDeviceToHost,
                         c->stream));
    }
  }
  CK(sync(c));
  loc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = loc;
  if (worst == IE_ENOCONV) c->err = "tolerance not reached within the iteration limits";
  return worst;
}

ie_status ie_solve_batch(int32_t n_items, ie_batch_item* items, int32_t max_concurrent) {
  if (n_items < 0 || (n_items > 0 && !items) || max_concurrent < 0) return IE_EINVAL;
  // group items by context, keeping the given order inside each group
  std::vector<ie_ctx*> ctxs;
  std::vector<std::vector<int>> groups;
  for (int i = 0; i < n_items; ++i) {
    items[i].status = IE_ESTATE;
    if (!items[i].ctx) {
      items[i].status = IE_EINVAL;
      continue;
    }
    size_t g = 0;
    while (g < ctxs.size() && ctxs[g] != items[i].ctx) ++g;
    if (g == ctxs.size()) {
      ctxs.push_back(items[i].ctx);
      groups.emplace_back();
    }
    groups[g].push_back(i);
  }
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return IE_ECUDA;
  // private non-blocking streams for contexts on the legacy default stream
  std::vector<cudaStream_t> owned(ctxs.size(), nullptr), saved(ctxs.size(), nullptr);
  for (size_t g = 0; g < ctxs.size(); ++g) {
    saved[g] = ctxs[g]->stream;
    if (!saved[g]) {
      DevGuard on_dev(ctxs[g]);
      if (!on_dev.ok || cudaStreamCreateWithFlags(&owned[g], cudaStreamNonBlocking) != cudaSuccess) {
        for (size_t h = 0; h < g; ++h)
          if (owned[h]) cudaStreamDestroy(owned[h]);
        return IE_ECUDA;
      }
      ctxs[g]->stream = owned[g];
    }
  }
  int workers = max_concurrent > 0 ? max_concurrent : (int)std::min<size_t>(ctxs.size(), 16);
  workers = std::max(1, std::min<int>(workers, (int)std::max<size_t>(ctxs.size(), 1)));
  std::atomic<int> next{0};
  auto work = [&]() {
    cudaSetDevice(device);
    for (int g; (g = next.fetch_add(1)) < (int)groups.size();) {
      for (int i : groups[g]) {
        ie_batch_item& it = items[i];
        it.status = it.sigma6 ? ie_set_contrast(it.ctx, it.sigma6) : IE_OK;
        if (it.status == IE_OK && it.E_init_dev) it.status = ie_set_initial_field_dev(it.ctx, it.E_init_dev);
        if (it.status == IE_OK)
          it.status = ie_solve(it.ctx, it.n_src, it.src, it.n_rx, it.rx_xyz, it.dd_mode, it.tol, it.opts, it.H_out,
                               it.info);
      }
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < workers; ++w) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
  for (size_t g = 0; g < ctxs.size(); ++g) {
    if (owned[g]) {
      DevGuard on_dev(ctxs[g]);
      cudaStreamSynchronize(owned[g]);
      cudaStreamDestroy(owned[g]);
      ctxs[g]->stream = saved[g];
    }
  }
  for (int i = 0; i < n_items; ++i)
    if (items[i].status != IE_OK) return items[i].status;
  return IE_OK;
}

ie_status ie_set_initial_field_dev(ie_ctx* c, const double* E_dev) {
  IE_ON_CTX_DEVICE(c);
  if (!c) return IE_EINVAL;
  if (!E_dev) {
    c->has_init = false;
    return IE_OK;
  }
  CK(c->Einit.ensure(sizeof(double2) * 3 * c->N));
  CK(cudaMemcpyAsync(c->Einit.p, E_dev, sizeof(double2) * 3 * c->N, cudaMemcpyDeviceToDevice, c->stream));
  c->has_init = true;
  return IE_OK;
}

ie_status ie_get_field_dev(ie_ctx* c, double* E_dev) {
  IE_ON_CTX_DEVICE(c);
  if (!c || !E_dev) return fail(c, IE_EINVAL, "null argument");
  if (!c->has_field) return fail(c, IE_ESTATE, "no solve has run");
  CK(cudaMemcpyAsync(E_dev, c->E.p, sizeof(double2) * 3 * c->N, cudaMemcpyDeviceToDevice, c->stream));
  return IE_OK;
}

ie_status ie_incident_field_dev(ie_ctx* c, const ie_dipole* src, double* E0_dev) {
  IE_ON_CTX_DEVICE(c);
  if (!c || !src || !E0_dev) return fail(c, IE_EINVAL, "null argument");
  CKS(check_point(c, src->pos));
  KL(IE_K_FIELD, 48.0 * c->N,
     launch_incident_E(reinterpret_cast<double2*>(E0_dev), c->nx, c->ny, c->nz, c->origin, c->h, src->pos,
                       src->moment, c->k0, c->omega * kMu0, c->stream));
  return IE_OK;
}

ie_status ie_get_field(ie_ctx* c, double* E_out) {
  IE_ON_CTX_DEVICE(c);
  if (!c || !E_out) return fail(c, IE_EINVAL, "null argument");
  if (!c->has_field) return fail(c, IE_ESTATE, "no solve has run");
  CK(cudaMemcpyAsync(E_out, c->E.p, sizeof(double2) * 3 * c->N, cudaMemcpyDeviceToHost, c->stream));
  CK(sync(c));
  return IE_OK;
}

ie_status ie_matvec(ie_ctx* c, int32_t precision, int32_t z0, int32_t nz, const double* x, double* y) {
  IE_ON_CTX_DEVICE(c);
  if (!c || !x || !y) return fail(c, IE_EINVAL, "null argument");
  const long nb = (long)nz * c->ny * c->nx;
  DevBuf xd, yd, xs, ys;
  CKS(upload_c128(c, x, 3 * std::max(nb, 0L), xd));
  if (precision == IE_PREC_FP64) {
    BlockOp<double> A;
    CKS(make_block<double>(c, z0, nz, &A));
    CK(yd.ensure(sizeof(double2) * 3 * nb));
    CKS(A.apply(xd.as<double2>(), yd.as<double2>()));
    CK(cudaMemcpyAsync(y, yd.p, sizeof(double2) * 3 * nb, cudaMemcpyDeviceToHost, c->stream));
  } else if (precision == IE_PREC_DFLOAT) {
    BlockOp<df> A;
    CKS(make_block<df>(c, z0, nz, &A));
    CK(yd.ensure(sizeof(double2) * 3 * nb));
    CKS(A.apply(xd.as<double2>(), yd.as<double2>()));
    CK(cudaMemcpyAsync(y, yd.p, sizeof(double2) * 3 * nb, cudaMemcpyDeviceToHost, c->stream));
  } else {
    BlockOp<float> A;
    CKS(make_block<float>(c, z0, nz, &A));
    CK(xs.ensure(sizeof(float2) * 3 * nb));
    CK(ys.ensure(sizeof(float2) * 3 * nb));
    CK(yd.ensure(sizeof(double2) * 3 * nb));
    KL(IE_K_FIELD, 72.0 * nb, launch_c128_to_c64(xd.as<double2>(), nb, xs.as<float2>(), nb, nb, c->stream));
    CKS(A.apply(xs.as<float2>(), ys.as<float2>()));
    CK(cudaMemsetAsync(yd.p, 0, sizeof(double2) * 3 * nb, c->stream));
    KL(IE_K_FIELD, 120.0 * nb, launch_add_c64_to_c128(ys.as<float2>(), nb, yd.as<double2>(), nb, nb, c->stream));
    CK(cudaMemcpyAsync(y, yd.p, sizeof(double2) * 3 * nb, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(sync(c));
  return IE_OK;
}

ie_status ie_matvec_contraction(ie_ctx* c, int32_t precision, int32_t z0, int32_t nz, const double* x, double* y) {
  IE_ON_CTX_DEVICE(c);
  if (!c || !x || !y) return fail(c, IE_EINVAL, "null argument");
  if (precision != IE_PREC_MIXED && precision != IE_PREC_FP64) return fail(c, IE_EINVAL, "bad precision");
  const long nb = (long)nz * c->ny * c->nx;
  DevBuf xd, yd, xs, ys;
  CKS(upload_c128(c, x, 3 * std::max(nb, 0L), xd));
  if (precision == IE_PREC_FP64) {
    BlockOp<double> A;
    CKS(make_block<double>(c, z0, nz, &A, true));
    CK(yd.ensure(sizeof(double2) * 3 * nb));
    CKS(A.apply(xd.as<double2>(), yd.as<double2>()));
  } else {
    BlockOp<float> A;
    CKS(make_block<float>(c, z0, nz, &A, true));
    CK(xs.ensure(sizeof(float2) * 3 * nb));
    CK(ys.ensure(sizeof(float2) * 3 * nb));
    CK(yd.ensure(sizeof(double2) * 3 * nb));
    KL(IE_K_FIELD, 72.0 * nb, launch_c128_to_c64(xd.as<double2>(), nb, xs.as<float2>(), nb, nb, c->stream));
    CKS(A.apply(xs.as<float2>(), ys.as<float2>()));
    CK(cudaMemsetAsync(yd.p, 0, sizeof(double2) * 3 * nb, c->stream));
    KL(IE_K_FIELD, 120.0 * nb, launch_add_c64_to_c128(ys.as<float2>(), nb, yd.as<double2>(), nb, nb, c->stream));
  }
  CK(cudaMemcpyAsync(y, yd.p, sizeof(double2) * 3 * nb, cudaMemcpyDeviceToHost, c->stream));
  CK(sync(c));
  return IE_OK;
}

ie_status ie_matvec_dev(ie_ctx* c, int32_t z0, int32_t nz, const void* x_dev, void* y_dev) {
  IE_ON_CTX_DEVICE(c);
  if (!c || !x_dev || !y_dev || x_dev == y_dev) return fail(c, IE_EINVAL, "bad argument");
  BlockOp<float> A;
  CKS(make_block<float>(c, z0, nz, &A));
  return A.apply(reinterpret_cast<const float2*>(x_dev), reinterpret_cast<float2*>(y_dev));
}

ie_status ie_interaction(ie_ctx* c, int32_t zs0, int32_t nzs, int32_t zt0, int32_t nzt, const double* x, double* y) {
  IE_ON_CTX_DEVICE(c);
  if (!c || !x || !y) return fail(c, IE_EINVAL, "null argument");
  if (zs0 < 0 || nzs < 1 || zs0 + nzs > c->nz || zt0 < 0 || nzt < 1 || zt0 + nzt > c->nz)
    return fail(c, IE_EINVAL, "slab outside the grid");
  if (!c->has_contrast) return fail(c, IE_ESTATE, "no contrast set");
  SpecSet* S = nullptr;
  CKS(get_spec(c, c->nz, &S));
  const long nxy = (long)c->nx * c->ny, ns = nzs * nxy, nt = nzt * nxy;
  DevBuf xd, yd;
  CKS(upload_c128(c, x, 3 * ns, xd));
  CK(yd.ensure(sizeof(double2) * 3 * nt));
  CKS(conv<double>(c, S, xd.as<double2>(), ns, zs0, nzs, zs0, nzt, zt0, EPI_CONV, nullptr, 0, yd.as<double2>(), nt,
                   nullptr, 0, nullptr, 0));
  CK(cudaMemcpyAsync(y, yd.p, sizeof(double2) * 3 * nt, cudaMemcpyDeviceToHost, c->stream));
  CK(sync(c));
  return IE_OK;
}

ie_status ie_gmres(ie_ctx* c, int32_t precision, int32_t z0, int32_t nz, const double* b, const double* x0, double tol,
                   int32_t restart, int32_t max_iter, double* x, int32_t* iters, double* rel) {
  IE_ON_CTX_DEVICE(c);
  if (!c || !b || !x || !(tol > 0) || max_iter < 0) return fail(c, IE_EINVAL, "bad argument");
  return precision == IE_PREC_FP64 ? gmres_host<double>(c, z0, nz, b, x0, tol, restart, max_iter, x, iters, rel)
                                   : gmres_host<float>(c, z0, nz, b, x0, tol, restart, max_iter, x, iters, rel);
}

ie_status ie_green_spectrum(ie_ctx* c, int32_t nz_set, int32_t comp, double* out, int32_t* dims) {
  IE_ON_CTX_DEVICE(c);
  if (!c || !out || comp < 0 || comp > 5 || nz_set < 1 || nz_set > c->nz) return fail(c, IE_EINVAL, "bad argument");
  SpecSet* S = nullptr;
  CKS(get_spec(c, nz_set, &S));
  const long ocs = (long)(c->Lx / 2 + 1) * (c->Ly / 2 + 1) * (S->Lz / 2 + 1);
  CK(cudaMemcpyAsync(out, S->G64.as<double2>() + comp * ocs, sizeof(double2) * ocs, cudaMemcpyDeviceToHost, c->stream));
  CK(sync(c));
  if (dims) {
    dims[0] = c->Lx;
    dims[1] = c->Ly;
    dims[2] = S->Lz;
  }
  return IE_OK;
}

ie_status ie_incident_field(ie_ctx* c, const ie_dipole* src, double* E0_out) {
  IE_ON_CTX_DEVICE(c);
  if (!c || !src || !E0_out) return fail(c, IE_EINVAL, "null argument");
  CKS(check_point(c, src->pos));
  DevBuf e;
  CK(e.ensure(sizeof(double2) * 3 * c->N));
  KL(IE_K_FIELD, 48.0 * c->N,
     launch_incident_E(e.as<double2>(), c->nx, c->ny, c->nz, c->origin, c->h, src->pos, src->moment, c->k0,
                       c->omega * kMu0, c->stream));
  CK(cudaMemcpyAsync(E0_out, e.p, sizeof(double2) * 3 * c->N, cudaMemcpyDeviceToHost, c->stream));
  CK(sync(c));
  return IE_OK;
}

ie_status ie_receiver_fields(ie_ctx* c, const double* E, const ie_dipole* src, int32_t n_rx, const double* rx,
                             double* H_out) {
  IE_ON_CTX_DEVICE(c);
  if (!c || !E || !src || (n_rx > 0 && (!rx || !H_out)) || n_rx < 0) return fail(c, IE_EINVAL, "bad argument");
  if (!c->has_contrast) return fail(c, IE_ESTATE, "no contrast set");
  for (int r = 0; r < n_rx; ++r) CKS(check_point(c, rx + 3 * r));
  if (n_rx == 0) return IE_OK;
  DevBuf ed, rxd, hd, pd;
  CKS(upload_c128(c, E, 3 * c->N, ed));
  CK(rxd.ensure(sizeof(double) * 3 * n_rx));
  CK(hd.ensure(sizeof(double2) * 3 * n_rx));
  CK(pd.ensure(sizeof(double2) * 3 * kMaxRx * receivers_partials_blocks(c->N)));
  CK(cudaMemcpyAsync(rxd.p, rx, sizeof(double) * 3 * n_rx, cudaMemcpyHostToDevice, c->stream));
  for (int r0 = 0; r0 < n_rx; r0 += kMaxRx) {
    const int nr = std::min(kMaxRx, n_rx - r0);
    KL(IE_K_FIELD, 96.0 * c->N,
       launch_receivers(ed.as<double2>(), c->N, c->ds64.as<double>(), c->N, c->nx, c->ny, c->origin, c->h,
                        rxd.as<double>() + 3 * r0, nr, c->k0, pd.as<double2>(), src->pos, src->moment,
                        hd.as<double2>() + 3 * r0, c->stream));
  }
  CK(cudaMemcpyAsync(H_out, hd.p, sizeof(double2) * 3 * n_rx, cudaMemcpyDeviceToHost, c->stream));
  CK(sync(c));
  return IE_OK;
}

ie_status ie_fft_dims(const ie_ctx* c, int32_t nz_set, int32_t* dims) {
  if (!c || !dims || nz_set < 1) return IE_EINVAL;
  dims[0] = c->Lx;
  dims[1] = c->Ly;
  dims[2] = next_pow2(2 * nz_set);
  return IE_OK;
}

ie_status ie_profile_enable(ie_ctx* c, int32_t on) {
  IE_ON_CTX_DEVICE(c);
  if (!c) return IE_EINVAL;
  CK(sync(c));
  auto& P = c->prof;
  P.on = on != 0;
  for (int k = 0; k < IE_K_COUNT; ++k) {
    P.launches[k] = 0;
    P.ms[k] = 0.0;
    P.bytes[k] = 0.0;
  }
  return IE_OK;
}

ie_status ie_profile_read(const ie_ctx* cc, int32_t kclass, int64_t* launches, double* ms, double* bytes) {
  if (!cc || kclass < 0 || kclass >= IE_K_COUNT) return IE_EINVAL;
  ie_ctx* c = const_cast<ie_ctx*>(cc);  // folding finished events into the counters is not observable state
  CK(drain(c));
  if (launches) *launches = c->prof.launches[kclass];
  if (ms) *ms = c->prof.ms[kclass];
  if (bytes) *bytes = c->prof.bytes[kclass];
  return IE_OK;
}

int32_t ie_tuned_tiles(char* buf, int32_t len) {
  std::string txt;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    static const char* pass[] = {"", "", "P2", "P3", "P4"};
    for (const auto& kv : g_tuned) {
      const TuneKey& k = kv.first;
      txt += std::string(pass[k.kind]) + " bytes=" + std::to_string(k.bytes) + " L=" + std::to_string(k.L) +
             " Lx=" + std::to_string(k.Lx) + " Ly=" + std::to_string(k.Ly) + " nz=" + std::to_string(k.nz) + "/" +
             std::to_string(k.nz2) + " variant=" + std::to_string(kv.second) + " us=";
      const auto it = g_tune_ms.find(k);
      if (it != g_tune_ms.end())
        for (size_t v = 0; v < it->second.size(); ++v)
          txt += (v ? "/" : "") + (std::isfinite(it->second[v])
                                         ? std::to_string((int)std::lround(1000.0 * it->second[v]))
                                         : std::string("-"));  // a variant this arithmetic does not build
      txt += "\n";
    }
  }
  if (buf && len > 0) {
    const size_t n = std::min<size_t>(txt.size(), (size_t)len - 1);
    std::memcpy(buf, txt.data(), n);
    buf[n] = 0;
  }
  return (int32_t)txt.size() + 1;
}

void ie_debug_fail_allocation(int32_t after) { g_alloc_fail_countdown.store(after < 0 ? -1 : after); }

ie_status ie_debug_force_tile(int32_t pass, int32_t variant) {
  if (pass < 2 || pass > 4) return IE_EINVAL;
  const int nvar = pass == 3 ? kP3TileVariants : kTileVariants;
  if (variant < -1 || variant >= nvar) return IE_EINVAL;
  g_force_tile[pass].store(variant);
  return IE_OK;
}

const char* ie_last_error(const ie_ctx* c) { return c ? c->err.c_str() : "null context"; }

void ie_destroy(ie_ctx* c) {
  if (!c) return;
  DevGuard on_dev(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  delete c;
}

}  // extern "C"

// =============================================================================== no-allocation operator
// Scratch of ie_matvec_dev_noalloc: the x-transformed (A) and xy-transformed (B) intermediates of the
// five FFT passes live in this fixed device array instead of context workspaces, so the call never
// allocates. Every GPU that loads the library reserves it for the life of the process.
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

// Device address of the scratch array on device `dev`, looked up once per device. The caller has made
// `dev` current (every entry point runs on its context's device), which is what the lookup needs: the
// array's host-side name is only a stand-in, and each device holds its own copy.
cudaError_t noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return e;
  if (cur != dev) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" ie_status ie_matvec_dev_noalloc(ie_ctx* c, int32_t z0, int32_t nz, const void* x_dev, void* y_dev) {
  IE_ON_CTX_DEVICE(c);
  if (!c || !x_dev || !y_dev || x_dev == y_dev) return fail(c, IE_EINVAL, "bad argument");
  if (z0 < 0 || nz < 1 || z0 + nz > c->nz) return fail(c, IE_EINVAL, "slab outside the grid");
  if (!c->has_contrast) return fail(c, IE_ESTATE, "no contrast set");
  const SpecSet* S = nullptr;
  for (auto* sp : c->specs)
    if (sp->nz_set == nz) S = sp;
  if (!S)
    return fail(c, IE_ESTATE,
                "no Green spectra for this slab height yet: ie_create prepares the whole grid; other heights are "
                "prepared by one ie_matvec_dev or ie_solve call first");
  const size_t a_bytes = sizeof(float2) * 3 * (size_t)nz * c->ny * c->Lx;
  const size_t b_off = (a_bytes + 255) & ~size_t(255);
  const size_t need = b_off + sizeof(float2) * 3 * (size_t)nz * c->Ly * c->Lx;
  if (need > kNoAllocScratchBytes)
    return fail(c, IE_EINVAL,
                "slab needs " + std::to_string(need) + " bytes of scratch, above the " +
                    std::to_string(kNoAllocScratchBytes) + "-byte limit of the no-allocation operator");
  void* base = nullptr;
  CK(noalloc_scratch(c->dev, &base));
  float2* A = reinterpret_cast<float2*>(base);
  float2* B = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(base) + b_off);
  const float2* x = reinterpret_cast<const float2*>(x_dev);
  float2* y = reinterpret_cast<float2*>(y_dev);
  const long nb = (long)nz * c->ny * c->nx, nxy = (long)c->nx * c->ny;
  const long A_cs = (long)nz * c->ny * c->Lx, B_cs = (long)nz * c->Ly * c->Lx;
  const float2* tw = c->tw32.as<float2>();
  cudaStream_t s = c->stream;
  // the five passes of the sub-domain operator; every scratch element they read was written first,
  // so nothing needs clearing between calls
  CK(ConvLaunch<float>::p1(c->Lx, x, nb, c->ds32.as<float>() + (long)z0 * nxy, c->N, A, A_cs, c->nx,
                           (long)nz * c->ny, tw, s));
  CK(ConvLaunch<float>::lanes(c->Ly, -1, 0, A, A_cs, (long)c->ny * c->Lx, c->Lx, c->ny, B, B_cs, (long)c->Ly * c->Lx,
                              c->Lx, c->Ly, c->Lx, nz, 3, tw, s));
  CK(ConvLaunch<float>::p3(S->Lz, 0, B, B_cs, nz, 0, B, B_cs, nz, 0, S->G32.as<float2>(), c->Lx, c->Ly, tw, c->kerr,
                           s));
  CK(ConvLaunch<float>::lanes(c->Ly, +1, 0, B, B_cs, (long)c->Ly * c->Lx, c->Lx, c->Ly, A, A_cs, (long)c->ny * c->Lx,
                              c->Lx, c->ny, c->Lx, nz, 3, tw, s));
  CK(ConvLaunch<float>::p5(c->Lx, EPI_APPLY, A, A_cs, c->nx, (long)nz * c->ny, x, nb, y, nb, nullptr, 0, nullptr, 0,
                           tw, s));
  return IE_OK;
}
