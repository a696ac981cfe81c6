// Host side of the C ABI declared in include/mg.h: context set-up, the sweep
// schedule (pass YZ, pass X, shell draw per sweep; captured into a CUDA graph),
// reads and writes of chain state, and error handling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mg.h"
#include "mg_aux.cuh"
#include "mg_launch.h"
#include "mg_persist.h"

#include <mutex>

using namespace mg;

namespace {

constexpr int kMaxBins = 254;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

struct Group {
  int n = 0;
  double L = 0;
  int B = 0;
  uint64_t seed = 0;
  double tau = 0;
  size_t M = 0;
  std::vector<long long> n_b;  // B+1
  std::shared_ptr<DevBuf> bc, bin_of_m2, n_b_dev, gamma, row_info, bc_rows;
  uint32_t bc_rows_len = 0;  // complex entries in bc_rows
};

struct Chain {
  int group = 0;
  uint32_t chain_id = 0;
  std::shared_ptr<DevBuf> main, nyq, coef, mscale, partial, P, sig, chi;
  std::shared_ptr<DevBuf> s1, s2;  // [M] FP64 sums of the recorded samples of s and of s^2
  std::shared_ptr<DevBuf> rec_desc;  // the chain's descriptor with the scratch field as output
  std::shared_ptr<DevBuf> trace;  // [records][B+1] P after every record_every-th sweep
  long long trace_cap = 0;        // records the trace buffer holds
};

// All chains of one grid size are launched together.
struct SizeClass {
  int n = 0;
  int C = 1;
  int B_max = 0;
  std::vector<int> chains;         // context chain indices
  std::shared_ptr<DevBuf> d_desc;  // ChainDev<T>[chains.size()]
  std::vector<char> h_desc;        // host copy of d_desc
  std::shared_ptr<DevBuf> tw;      // twiddle tables (TwLayout), context precision
  std::vector<std::vector<char>> args;  // LaunchArgs<T> per chunk of <= kMaxLaunchChains chains
};

// Work buffers of mg_adjoint for one grid size, kept between calls.
struct AdjWork {
  int K_cap = 0;  // checkpoints ck holds
  int B1 = 0;     // shells + 1 that acc and Psave hold
  std::shared_ptr<DevBuf> ck, scr, adj, wl64, wl, dd, ddw, acc, Psave, desc, sw;
  cudaStream_t up = nullptr;  // the loss weights' upload, beside the forward sweeps
  cudaEvent_t up_ev = nullptr;
  AdjWork() = default;
  AdjWork(const AdjWork&) = delete;
  AdjWork& operator=(const AdjWork&) = delete;
  ~AdjWork() {
    if (up_ev) cudaEventDestroy(up_ev);
    if (up) cudaStreamDestroy(up);
  }
};

}  // namespace

struct mg_ctx {
  int precision = 64;
  int fix_P = 0;
  int mixing = 0;  // 1: every sweep uses the mixing sampler (Sec. 3.3); 2: odd sweeps do
  int record_every = 0;
  long long records = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<Group> groups;
  std::vector<Chain> chains;
  std::vector<SizeClass> classes;
  std::shared_ptr<DevBuf> d_draw;  // DrawDev[chains]
  std::shared_ptr<DevBuf> d_sweep, d_status, d_scratch_s;
  std::shared_ptr<DevBuf> d_pk_all;  // staging of mg_read_pk_all
  std::shared_ptr<DevBuf> d_rec_now;  // int: the next pass YZ adds its incoming state to the sums
  bool stats_pending = false;         // the current state is a recorded sample not yet in the sums
  std::map<int, AdjWork> adj_work;   // mg_adjoint's buffers per grid size
  int B_max = 0;
  long long sweeps = 0;
  mg_status sticky = MG_OK;
  std::string err;
  // one stream per grid size beyond the first, so that the size classes'
  // passes of a sweep run as parallel branches (fork and join by events)
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> aux_ev;  // [0] fork, [1 + k] join of class k
  cudaGraphExec_t graph = nullptr;      // one plain sweep
  cudaGraphExec_t graph_mix = nullptr;  // one mixing sweep
  bool graph_failed = false;
  // persistent one-launch sweep
  bool persist = false;
  std::vector<char> persist_args;  // PersistArgs<T>
  std::shared_ptr<DevBuf> persist_ctr;
  int persist_grid = 0;
  long long timeout = 0;
  int fault_in = 0;  // mg_inject_cuda_error: checked CUDA calls left until a faked failure (0: off)
};

namespace {

thread_local std::string g_create_error;  // why the last mg_init / mg_init_batch failed

mg_status fail(mg_ctx* c, mg_status s, const std::string& msg) {
  g_create_error = msg;
  if (c) {
    c->err = msg;
    if (s == MG_ECUDA || s == MG_ENUMERIC || s == MG_ETIMEOUT || s == MG_EBOUNDS) c->sticky = s;
  }
  return s;
}

// Host-side fault injection (mg_inject_cuda_error): the checked CUDA call that
// brings the context's countdown to zero is not made and reports
// cudaErrorUnknown instead, as a failing call would.
bool fake_cuda_fault(mg_ctx* c) {
  if (!c || c->fault_in <= 0) return false;
  return --c->fault_in == 0;
}

#define MG_CUDA(ctx, call)                                                                  \
  do {                                                                                      \
    const bool fake_ = fake_cuda_fault(ctx);                                                \
    cudaError_t e_ = fake_ ? cudaErrorUnknown : (call);                                     \
    if (e_ != cudaSuccess)                                                                  \
      return fail(ctx, MG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_) +       \
                                     (fake_ ? " (injected by mg_inject_cuda_error)" : "")); \
  } while (0)

std::shared_ptr<DevBuf> dalloc(size_t bytes, cudaError_t* err) {
  auto b = std::make_shared<DevBuf>();
  b->bytes = bytes;
  *err = cudaMalloc(&b->p, bytes ? bytes : 16);
  if (*err != cudaSuccess) b->p = nullptr;
  return b;
}

bool is_supported_n(int n) {
  static const int ok[] = {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256};
  for (int v : ok)
    if (v == n) return n <= MG_MAX_N;
  return false;
}

// Shell id of every |m|^2 (host, once per group).  Linear edges use the exact
// integer test b^2 (n/2)^2 <= B^2 m^2 (ties go to the upper shell); explicit
// edges compare |k| = (2 pi / L) sqrt(m^2) in FP64.  Out-of-range -> B.
std::vector<uint8_t> build_bin_table(int n, double L, int B, const double* edges, std::vector<long long>* n_b) {
  const int h = n / 2;
  const int max_m2 = 3 * h * h;
  std::vector<uint8_t> tab(size_t(max_m2) + 1, uint8_t(B));
  for (int m2 = 1; m2 <= max_m2; ++m2) {
    int b;
    if (!edges) {
      // largest b with b^2 h^2 <= B^2 m2: b = floor(sqrt(B^2 m2) / h), exact
      const unsigned long long t = (unsigned long long)B * B * (unsigned long long)m2;
      unsigned long long q = (unsigned long long)std::sqrt((double)t);
      while (q * q > t) --q;
      while ((q + 1) * (q + 1) <= t) ++q;
      b = int(q / (unsigned long long)h);
      if (b >= B) b = B;
    } else {
      const double k = 2.0 * M_PI / L * std::sqrt(double(m2));
      b = -1;
      for (int e = 0; e < B; ++e)
        if (k >= edges[e]) b = e;
      if (b < 0 || k >= edges[B]) b = B;
    }
    tab[m2] = uint8_t(b);
  }
  // full-grid mode counts per shell: the modes with |m|^2 = m2 counted over
  // the distinct |m| of each axis, weighted by how many k give that |m|
  n_b->assign(B + 1, 0);
  std::vector<long long> cnt(size_t(max_m2) + 1, 0);
  std::vector<long long> mult(size_t(h) + 1, 0);
  for (int k = 0; k < n; ++k) ++mult[std::abs(k <= h ? k : k - n)];
  for (int a = 0; a <= h; ++a)
    for (int b2 = 0; b2 <= h; ++b2) {
      const long long wab = mult[a] * mult[b2];
      const int s2 = a * a + b2 * b2;
      for (int c = 0; c <= h; ++c) cnt[s2 + c * c] += wab * mult[c];
    }
  for (int m2 = 1; m2 <= max_m2; ++m2) (*n_b)[tab[m2]] += cnt[m2];
  return tab;
}

void split_of(int n, int* P, int* Q) {
  switch (n) {
#define MG_SPLIT_CASE(N_) \
  case N_:                \
    *P = Split<N_>::P;    \
    *Q = Split<N_>::Q;    \
    return;
    MG_SPLIT_CASE(4)
    MG_SPLIT_CASE(6)
    MG_SPLIT_CASE(8)
    MG_SPLIT_CASE(12)
    MG_SPLIT_CASE(16)
    MG_SPLIT_CASE(24)
    MG_SPLIT_CASE(32)
    MG_SPLIT_CASE(48)
    MG_SPLIT_CASE(64)
    MG_SPLIT_CASE(96)
    MG_SPLIT_CASE(128)
    MG_SPLIT_CASE(192)
    MG_SPLIT_CASE(256)
#undef MG_SPLIT_CASE
    default:
      *P = *Q = 0;
  }
}

// Twiddle tables of grid size n in the layout of TwLayout (mg_device.cuh),
// each value exp(-2 pi i e / n) evaluated in long double and rounded once.
template <typename T>
std::vector<typename VT<T>::c2> twiddles(int n) {
  int P, Q, P2, Q2;
  split_of(n, &P, &Q);
  split_of(n / 2, &P2, &Q2);
  std::vector<typename VT<T>::c2> t(size_t(4) * n + n / 2);
  auto W = [n](long e) {
    const long double a = -2.0L * 3.14159265358979323846264338327950288L * (long double)(e % n) / (long double)n;
    typename VT<T>::c2 v;
    v.x = T(std::cos(a));
    v.y = T(std::sin(a));
    return v;
  };
  for (int k = 0; k < n; ++k) t[k] = W(k);
  for (int v = 0; v < Q; ++v)
    for (int p = 0; p < P; ++p) {
      t[n + v * P + p] = W(long(p) * v);
      t[2 * n + p * Q + v] = W(long(p) * v);
    }
  for (int v = 0; v < Q2; ++v)
    for (int p = 0; p < P2; ++p) {
      t[3 * n + v * P2 + p] = W(2L * p * v);
      t[3 * n + n / 2 + p * Q2 + v] = W(2L * p * v);
      t[4 * n + v * P2 + p] = W(long(Q2) * p + v);
    }
  return t;
}

template <typename T>
mg_status upload_descriptors(mg_ctx* c) {
  using V2 = typename VT<T>::c2;
  for (auto& sc : c->classes) {
    std::vector<ChainDev<T>> h(sc.chains.size());
    for (size_t i = 0; i < sc.chains.size(); ++i) {
      const Chain& ch = c->chains[sc.chains[i]];
      const Group& g = c->groups[ch.group];
      ChainDev<T>& d = h[i];
      d.main = static_cast<V2*>(ch.main->p);
      d.nyq = static_cast<V2*>(ch.nyq->p);
      d.row_info = static_cast<const uint2*>(g.row_info->p);
      d.bc_rows = static_cast<const V2*>(g.bc_rows->p);
      d.coef = static_cast<const V2*>(ch.coef->p);
      d.mscale = static_cast<const T*>(ch.mscale->p);
      d.partial = static_cast<double*>(ch.partial->p);
      d.bin_of_m2 = static_cast<const uint8_t*>(g.bin_of_m2->p);
      d.s1 = ch.s1 ? static_cast<double*>(ch.s1->p) : nullptr;
      d.s2 = ch.s2 ? static_cast<double*>(ch.s2->p) : nullptr;
      d.s_out = nullptr;
      d.s_in = nullptr;
      d.status = static_cast<int*>(c->d_status->p);
      d.bc_rows_len = g.bc_rows_len;
      d.tau = T(g.tau);
      d.B = g.B;
    }
    cudaError_t e;
    sc.d_desc = dalloc(h.size() * sizeof(ChainDev<T>), &e);
    MG_CUDA(c, e);
    MG_CUDA(c, cudaMemcpyAsync(sc.d_desc->p, h.data(), h.size() * sizeof(ChainDev<T>), cudaMemcpyHostToDevice, c->stream));
    sc.h_desc.assign(reinterpret_cast<const char*>(h.data()), reinterpret_cast<const char*>(h.data() + h.size()));
    const auto tw = twiddles<T>(sc.n);
    sc.tw = dalloc(tw.size() * sizeof(V2), &e);
    MG_CUDA(c, e);
    MG_CUDA(c, cudaMemcpyAsync(sc.tw->p, tw.data(), tw.size() * sizeof(V2), cudaMemcpyHostToDevice, c->stream));
    sc.args.clear();
    for (size_t c0 = 0; c0 < sc.chains.size(); c0 += kMaxLaunchChains) {
      LaunchArgs<T> a;
      std::memset(&a, 0, sizeof(a));
      a.chains = static_cast<const ChainDev<T>*>(sc.d_desc->p) + c0;
      a.sweep_ctr = static_cast<const uint32_t*>(c->d_sweep->p);
      a.tw = static_cast<const V2*>(sc.tw->p);
      a.rec_now = static_cast<const int*>(c->d_rec_now->p);
      a.n_chains = int(std::min<size_t>(kMaxLaunchChains, sc.chains.size() - c0));
      for (int k = 0; k < a.n_chains; ++k) {
        const Chain& ch = c->chains[sc.chains[c0 + k]];
        const Group& g = c->groups[ch.group];
        a.k0[k] = uint32_t(g.seed & 0xffffffffu);
        a.k1[k] = uint32_t(g.seed >> 32);
        a.cid[k] = ch.chain_id;
      }
      sc.args.emplace_back(reinterpret_cast<const char*>(&a), reinterpret_cast<const char*>(&a) + sizeof(a));
    }
  }
  std::vector<DrawDev> dd(c->chains.size());
  for (size_t i = 0; i < c->chains.size(); ++i) {
    const Chain& ch = c->chains[i];
    const Group& g = c->groups[ch.group];
    DrawDev& d = dd[i];
    d.partial = static_cast<const double*>(ch.partial->p);
    d.n_tiles = pass_x_tiles(g.n);
    d.B = g.B;
    d.n_b = static_cast<const long long*>(g.n_b_dev->p);
    d.P = static_cast<double*>(ch.P->p);
    d.sig_last = static_cast<double*>(ch.sig->p);
    d.chi_last = static_cast<double*>(ch.chi->p);
    d.coef = ch.coef->p;
    d.mscale = ch.mscale->p;
    d.k0 = uint32_t(g.seed & 0xffffffffu);
    d.k1 = uint32_t(g.seed >> 32);
    d.cid = ch.chain_id;
    d.tau = g.tau;
    d.M = double(g.M);
    d.V = g.L * g.L * g.L;
  }
  cudaError_t e;
  c->d_draw = dalloc(dd.size() * sizeof(DrawDev), &e);
  MG_CUDA(c, e);
  MG_CUDA(c, cudaMemcpyAsync(c->d_draw->p, dd.data(), dd.size() * sizeof(DrawDev), cudaMemcpyHostToDevice, c->stream));
  return MG_OK;
}

template <typename T>
mg_status launch_shell_draw(mg_ctx* c, int draw, bool count_sweep) {
  const dim3 grid(unsigned(c->chains.size()), unsigned(c->B_max + 1));
  shell_draw_kernel<T><<<grid, 256, 0, c->stream>>>(static_cast<const DrawDev*>(c->d_draw->p), draw, c->fix_P,
                                                    static_cast<int*>(c->d_status->p),
                                                    count_sweep ? static_cast<uint32_t*>(c->d_sweep->p) : nullptr);
  MG_CUDA(c, cudaGetLastError());
  return MG_OK;
}

// Run fn(size class, stream) for every size class: in order on the context's
// stream for one class, else as parallel branches forked from and joined
// back into it (in a captured sweep they become parallel graph branches).
template <typename F>
mg_status for_each_class(mg_ctx* c, F fn) {
  if (c->classes.size() < 2) {
    for (auto& sc : c->classes) {
      mg_status st = fn(sc, c->stream);
      if (st != MG_OK) return st;
    }
    return MG_OK;
  }
  const size_t K = c->classes.size();
  while (c->aux.size() < K) {
    cudaStream_t st;
    MG_CUDA(c, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    c->aux.push_back(st);
  }
  while (c->aux_ev.size() < K + 1) {
    cudaEvent_t ev;
    MG_CUDA(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    c->aux_ev.push_back(ev);
  }
  MG_CUDA(c, cudaEventRecord(c->aux_ev[0], c->stream));
  for (size_t k = 0; k < K; ++k) {
    MG_CUDA(c, cudaStreamWaitEvent(c->aux[k], c->aux_ev[0], 0));
    mg_status st = fn(c->classes[k], c->aux[k]);
    if (st != MG_OK) return st;
    MG_CUDA(c, cudaEventRecord(c->aux_ev[1 + k], c->aux[k]));
  }
  for (size_t k = 0; k < K; ++k) MG_CUDA(c, cudaStreamWaitEvent(c->stream, c->aux_ev[1 + k], 0));
  return MG_OK;
}

// Recorded samples are added to the sums inside the next sweep's pass YZ
// (its record mode), except under the persistent schedule, which adds them
// with a separate pass right after the sweep.
bool fused_record(const mg_ctx* c) { return c->record_every > 0 && !c->persist; }

// which: bit 1 = pass YZ of every size class, bit 2 = pass X, bit 4 = shell draw.
// A whole sweep (which = 7) runs each size class's passes as its own branch.
template <typename T>
mg_status enqueue_passes(mg_ctx* c, int which, bool mix) {
  const int yz_mode = fused_record(c) ? int(kModeSweepRecord) : int(kModeSweep);
  auto yz = [c, yz_mode](SizeClass& sc, cudaStream_t st) -> mg_status {
    for (auto& blob : sc.args)
      MG_CUDA(c, launch_pass_yz<T>(sc.n, sc.C, yz_mode, *reinterpret_cast<const LaunchArgs<T>*>(blob.data()), st));
    return MG_OK;
  };
  auto xpass = [c](int mode) {
    return [c, mode](SizeClass& sc, cudaStream_t st) -> mg_status {
      for (auto& blob : sc.args)
        MG_CUDA(c, launch_pass_x<T>(sc.n, mode, *reinterpret_cast<const LaunchArgs<T>*>(blob.data()), sc.B_max, st));
      return MG_OK;
    };
  };
  if (which == 7) {
    mg_status st;
    if (mix) {
      auto first = [&](SizeClass& sc, cudaStream_t s) -> mg_status {
        mg_status r = yz(sc, s);
        return r != MG_OK ? r : xpass(kXMixDraw)(sc, s);
      };
      if ((st = for_each_class(c, first)) != MG_OK) return st;
      const dim3 grid(unsigned(c->chains.size()), unsigned(c->B_max + 1));
      mixing_draw_kernel<T><<<grid, 256, 0, c->stream>>>(static_cast<const DrawDev*>(c->d_draw->p),
                                                         static_cast<int*>(c->d_status->p),
                                                         static_cast<const uint32_t*>(c->d_sweep->p));
      MG_CUDA(c, cudaGetLastError());
      if ((st = for_each_class(c, xpass(kXMixScale))) != MG_OK) return st;
      sweep_bump_kernel<<<1, 1, 0, c->stream>>>(static_cast<uint32_t*>(c->d_sweep->p));
      MG_CUDA(c, cudaGetLastError());
      return MG_OK;
    }
    auto both = [&](SizeClass& sc, cudaStream_t s) -> mg_status {
      mg_status r = yz(sc, s);
      return r != MG_OK ? r : xpass(0)(sc, s);
    };
    if ((st = for_each_class(c, both)) != MG_OK) return st;
    return launch_shell_draw<T>(c, 1, true);
  }
  if (which & 1) {
    for (auto& sc : c->classes)
      for (auto& blob : sc.args)
        MG_CUDA(c, launch_pass_yz<T>(sc.n, sc.C, yz_mode, *reinterpret_cast<const LaunchArgs<T>*>(blob.data()),
                                     c->stream));
  }
  if (mix) {
    // mixing sweep: x draw and its shell sums (modes left in k space), the
    // Metropolis-Hastings step per shell, the rescale and inverse x FFT; the
    // sweep counter advances last
    if (which & 2) {
      for (auto& sc : c->classes)
        for (auto& blob : sc.args)
          MG_CUDA(c, launch_pass_x<T>(sc.n, kXMixDraw, *reinterpret_cast<const LaunchArgs<T>*>(blob.data()),
                                      sc.B_max, c->stream));
      const dim3 grid(unsigned(c->chains.size()), unsigned(c->B_max + 1));
      mixing_draw_kernel<T><<<grid, 256, 0, c->stream>>>(static_cast<const DrawDev*>(c->d_draw->p),
                                                         static_cast<int*>(c->d_status->p),
                                                         static_cast<const uint32_t*>(c->d_sweep->p));
      MG_CUDA(c, cudaGetLastError());
      for (auto& sc : c->classes)
        for (auto& blob : sc.args)
          MG_CUDA(c, launch_pass_x<T>(sc.n, kXMixScale, *reinterpret_cast<const LaunchArgs<T>*>(blob.data()),
                                      sc.B_max, c->stream));
    }
    if (which & 4) {
      sweep_bump_kernel<<<1, 1, 0, c->stream>>>(static_cast<uint32_t*>(c->d_sweep->p));
      MG_CUDA(c, cudaGetLastError());
    }
    return MG_OK;
  }
  if (which & 2) {
    for (auto& sc : c->classes)
      for (auto& blob : sc.args)
        MG_CUDA(c, launch_pass_x<T>(sc.n, 0, *reinterpret_cast<const LaunchArgs<T>*>(blob.data()), sc.B_max, c->stream));
  }
  if (which & 4) return launch_shell_draw<T>(c, 1, true);
  return MG_OK;
}

bool persist_eligible(const mg_ctx* c) {
  if (c->classes.empty() || c->classes.size() > size_t(kMaxPersistClasses)) return false;
  for (const auto& sc : c->classes)
    if (!persist_supports(sc.n) || sc.C != 1 || sc.chains.size() > size_t(kMaxLaunchChains)) return false;
  return true;
}

// Build the persistent launch's parameters (queue layout, chain numbering).
template <typename T>
mg_status build_persist(mg_ctx* c) {
  PersistArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.ncls = int(c->classes.size());
  int u = 0;
  for (int k = 0; k < a.ncls; ++k) {
    const SizeClass& sc = c->classes[k];
    a.cls[k] = *reinterpret_cast<const LaunchArgs<T>*>(sc.args[0].data());
    a.n[k] = sc.n;
    a.tiles[k] = pass_x_tiles(sc.n);
    for (size_t i = 0; i < sc.chains.size(); ++i) a.ctx_chain[k][i] = sc.chains[i];
    a.yz_begin[k] = u;
    u += sc.n * int(sc.chains.size());
  }
  a.yz_begin[a.ncls] = u;
  for (int k = 0; k < a.ncls; ++k) {
    a.x_begin[k] = u;
    u += a.tiles[k] * int(c->classes[k].chains.size());
  }
  a.x_begin[a.ncls] = u;
  a.draw_begin = u;
  a.n_chains_total = int(c->chains.size());
  a.total = u + a.n_chains_total;
  a.fix_P = c->fix_P;
  a.timeout = c->timeout;
  cudaError_t e;
  c->persist_ctr = dalloc(size_t(2 + 2 * a.n_chains_total) * sizeof(unsigned), &e);
  MG_CUDA(c, e);
  a.ctr = static_cast<unsigned*>(c->persist_ctr->p);
  a.draw = static_cast<const DrawDev*>(c->d_draw->p);
  a.status = static_cast<int*>(c->d_status->p);
  a.sweep_ctr = static_cast<uint32_t*>(c->d_sweep->p);
  c->persist_grid = persist_grid<T>(a, c->B_max);
  if (c->persist_grid <= 0) return fail(c, MG_ECUDA, "persistent kernel does not fit on this GPU");
  c->persist_args.assign(reinterpret_cast<const char*>(&a), reinterpret_cast<const char*>(&a) + sizeof(a));
  return MG_OK;
}

template <typename T>
mg_status enqueue_persistent(mg_ctx* c) {
  const auto& a = *reinterpret_cast<const PersistArgs<T>*>(c->persist_args.data());
  MG_CUDA(c, cudaMemsetAsync(c->persist_ctr->p, 0, size_t(2 + 2 * a.n_chains_total) * sizeof(unsigned), c->stream));
  MG_CUDA(c, launch_persistent<T>(a, c->B_max, c->persist_grid, c->stream));
  return MG_OK;
}

// Whether the context's next sweep is a mixing sweep (the sweep count is the
// Philox counter word of that sweep).
bool mixing_sweep_next(const mg_ctx* c) { return c->mixing == 1 || (c->mixing == 2 && (c->sweeps & 1)); }

mg_status enqueue_sweep(mg_ctx* c, bool mix) {
  if (c->persist) return c->precision == 32 ? enqueue_persistent<float>(c) : enqueue_persistent<double>(c);
  return c->precision == 32 ? enqueue_passes<float>(c, 7, mix) : enqueue_passes<double>(c, 7, mix);
}

void drop_graph(mg_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->graph_mix) cudaGraphExecDestroy(c->graph_mix);
  c->graph = nullptr;
  c->graph_mix = nullptr;
  c->graph_failed = false;
}

// ---------------------------------------------------------------------------
// Autotuner: time the schedules the build provides on the context's own
// chains (state saved and restored around every trial) and keep the fastest.
// ---------------------------------------------------------------------------

mg_status check_status(mg_ctx* c);

struct Schedule {
  std::vector<int> C;
  bool persist = false;
};
std::mutex g_tune_mu;
std::map<std::string, Schedule> g_tune_cache;

std::string tune_key(const mg_ctx* c) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, dev);
  std::string k = std::string(prop.name) + "|" + std::to_string(c->precision) + (c->mixing ? "|mix" : "");
  for (const auto& sc : c->classes) k += "|" + std::to_string(sc.n) + "x" + std::to_string(sc.chains.size());
  return k;
}

mg_status flush_stats(mg_ctx* c);

template <typename T>
mg_status tune_impl(mg_ctx* c, int reps) {
  using V2 = typename VT<T>::c2;
  if (reps < 1) reps = 1;
  {
    // the trial sweeps must not add anything to the sums
    const mg_status fs = flush_stats(c);
    if (fs != MG_OK) return fs;
    MG_CUDA(c, cudaMemsetAsync(c->d_rec_now->p, 0, sizeof(int), c->stream));
  }
  const std::string key = tune_key(c);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      for (size_t k = 0; k < c->classes.size(); ++k) c->classes[k].C = it->second.C[k];
      c->persist = false;
      if (it->second.persist && !c->mixing) {
        mg_status st = build_persist<T>(c);
        if (st != MG_OK) return st;
        c->persist = true;
      }
      drop_graph(c);
      return MG_OK;
    }
  }
  cudaStream_t s = c->stream;
  // save every chain's state, P and the sweep counter
  std::vector<std::shared_ptr<DevBuf>> save(c->chains.size());
  std::vector<size_t> main_b(c->chains.size()), nyq_b(c->chains.size()), p_b(c->chains.size());
  cudaError_t e;
  for (size_t i = 0; i < c->chains.size(); ++i) {
    const Group& g = c->groups[c->chains[i].group];
    main_b[i] = size_t(g.n) * g.n * (g.n / 2) * sizeof(V2);
    nyq_b[i] = size_t(g.n) * g.n * sizeof(V2);
    p_b[i] = size_t(g.B + 1) * sizeof(double);
    save[i] = dalloc(main_b[i] + nyq_b[i] + p_b[i], &e);
    MG_CUDA(c, e);
    char* d = static_cast<char*>(save[i]->p);
    MG_CUDA(c, cudaMemcpyAsync(d, c->chains[i].main->p, main_b[i], cudaMemcpyDeviceToDevice, s));
    MG_CUDA(c, cudaMemcpyAsync(d + main_b[i], c->chains[i].nyq->p, nyq_b[i], cudaMemcpyDeviceToDevice, s));
    MG_CUDA(c, cudaMemcpyAsync(d + main_b[i] + nyq_b[i], c->chains[i].P->p, p_b[i], cudaMemcpyDeviceToDevice, s));
  }
  uint32_t sw0 = 0;
  MG_CUDA(c, cudaMemcpyAsync(&sw0, c->d_sweep->p, sizeof(sw0), cudaMemcpyDeviceToHost, s));
  MG_CUDA(c, cudaStreamSynchronize(s));
  auto restore = [&]() -> mg_status {
    for (size_t i = 0; i < c->chains.size(); ++i) {
      const char* d = static_cast<const char*>(save[i]->p);
      MG_CUDA(c, cudaMemcpyAsync(c->chains[i].main->p, d, main_b[i], cudaMemcpyDeviceToDevice, s));
      MG_CUDA(c, cudaMemcpyAsync(c->chains[i].nyq->p, d + main_b[i], nyq_b[i], cudaMemcpyDeviceToDevice, s));
      MG_CUDA(c, cudaMemcpyAsync(c->chains[i].P->p, d + main_b[i] + nyq_b[i], p_b[i], cudaMemcpyDeviceToDevice, s));
    }
    MG_CUDA(c, cudaMemcpyAsync(c->d_sweep->p, &sw0, sizeof(sw0), cudaMemcpyHostToDevice, s));
    mg_status st = launch_shell_draw<T>(c, 0, false);
    if (st != MG_OK) return st;
    MG_CUDA(c, cudaStreamSynchronize(s));
    return MG_OK;
  };
  cudaEvent_t e0, e1;
  MG_CUDA(c, cudaEventCreate(&e0));
  MG_CUDA(c, cudaEventCreate(&e1));
  auto elapsed = [&](float* ms) -> mg_status {
    MG_CUDA(c, cudaEventSynchronize(e1));
    MG_CUDA(c, cudaEventElapsedTime(ms, e0, e1));
    return MG_OK;
  };
  mg_status st = MG_OK;
  // 1. the y/z cluster size of each grid size, timing that pass alone
  for (auto& sc : c->classes) {
    int cand[4];
    const int nc = yz_cluster_choices(sc.n, c->precision, cand, 4);
    float best = 1e30f;
    int bestC = sc.C;
    for (int i = 0; i < nc; ++i) {
      LaunchArgs<T> none;
      std::memset(&none, 0, sizeof(none));
      MG_CUDA(c, launch_pass_yz<T>(sc.n, cand[i], 0, none, s));
      const LaunchArgs<T>& la = *reinterpret_cast<const LaunchArgs<T>*>(sc.args[0].data());
      for (auto& blob : sc.args)  // warm-up
        MG_CUDA(c, launch_pass_yz<T>(sc.n, cand[i], 0, *reinterpret_cast<const LaunchArgs<T>*>(blob.data()), s));
      (void)la;
      MG_CUDA(c, cudaEventRecord(e0, s));
      for (int r = 0; r < reps; ++r)
        for (auto& blob : sc.args)
          MG_CUDA(c, launch_pass_yz<T>(sc.n, cand[i], 0, *reinterpret_cast<const LaunchArgs<T>*>(blob.data()), s));
      MG_CUDA(c, cudaEventRecord(e1, s));
      float ms = 0.f;
      if ((st = elapsed(&ms)) != MG_OK) return st;
      if (ms < best) {
        best = ms;
        bestC = cand[i];
      }
      if ((st = restore()) != MG_OK) return st;
    }
    sc.C = bestC;
  }
  // 2. one persistent launch per sweep against one launch per pass
  c->persist = false;
  bool use_persist = false;
  if (!c->mixing && persist_eligible(c)) {
    if ((st = build_persist<T>(c)) != MG_OK) return st;
    float t[2];
    for (int mode = 0; mode < 2; ++mode) {
      c->persist = mode == 1;
      if ((st = enqueue_sweep(c, false)) != MG_OK) return st;  // warm-up
      MG_CUDA(c, cudaEventRecord(e0, s));
      for (int r = 0; r < reps; ++r)
        if ((st = enqueue_sweep(c, false)) != MG_OK) return st;
      MG_CUDA(c, cudaEventRecord(e1, s));
      if ((st = elapsed(&t[mode])) != MG_OK) return st;
      if ((st = restore()) != MG_OK) return st;
    }
    use_persist = t[1] < t[0];
  }
  c->persist = use_persist;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_graph(c);
  Schedule sch;
  for (const auto& sc : c->classes) sch.C.push_back(sc.C);
  sch.persist = use_persist;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = sch;
  return check_status(c);
}

// The size class of a chain and its index there (false if out of range).
bool find_chain(mg_ctx* c, int chain, SizeClass** sc, size_t* idx) {
  for (auto& k : c->classes)
    for (size_t i = 0; i < k.chains.size(); ++i)
      if (k.chains[i] == chain) {
        *sc = &k;
        *idx = i;
        return true;
      }
  return false;
}

// Launch arguments of one chain (n_chains = 1) with the descriptor `dev`.
template <typename T>
LaunchArgs<T> one_chain_args(const SizeClass& sc, size_t i, const ChainDev<T>* dev) {
  const LaunchArgs<T>& src = *reinterpret_cast<const LaunchArgs<T>*>(sc.args[i / kMaxLaunchChains].data());
  LaunchArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.chains = dev;
  a.sweep_ctr = src.sweep_ctr;
  a.tw = src.tw;
  a.rec_now = src.rec_now;
  a.n_chains = 1;
  a.k0[0] = src.k0[i % kMaxLaunchChains];
  a.k1[0] = src.k1[i % kMaxLaunchChains];
  a.cid[0] = src.cid[i % kMaxLaunchChains];
  return a;
}

// Launch arguments for one chain with an input or output field pointer
// attached (a descriptor of its own in *desc).
template <typename T>
mg_status single_chain_args(mg_ctx* c, int chain, T* s_out, const T* s_in, SizeClass** sc_out,
                            std::shared_ptr<DevBuf>* desc, LaunchArgs<T>* args) {
  SizeClass* sc;
  size_t i;
  if (!find_chain(c, chain, &sc, &i)) return fail(c, MG_EINVAL, "chain index out of range");
  ChainDev<T> h = reinterpret_cast<const ChainDev<T>*>(sc->h_desc.data())[i];
  h.s_out = s_out;
  h.s_in = s_in;
  cudaError_t e;
  *desc = dalloc(sizeof(h), &e);
  MG_CUDA(c, e);
  MG_CUDA(c, cudaMemcpyAsync((*desc)->p, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  *args = one_chain_args<T>(*sc, i, static_cast<const ChainDev<T>*>((*desc)->p));
  *sc_out = sc;
  return MG_OK;
}

template <typename T>
mg_status materialize(mg_ctx* c, int chain, T* out_dev) {
  SizeClass* sc;
  std::shared_ptr<DevBuf> desc;
  LaunchArgs<T> a;
  mg_status s = single_chain_args<T>(c, chain, out_dev, nullptr, &sc, &desc, &a);
  if (s != MG_OK) return s;
  MG_CUDA(c, launch_pass_yz<T>(sc->n, sc->C, 1, a, c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  return MG_OK;
}

template <typename T>
mg_status load_s(mg_ctx* c, int chain, const T* in_dev) {
  SizeClass* sc;
  std::shared_ptr<DevBuf> desc;
  LaunchArgs<T> a;
  mg_status s = single_chain_args<T>(c, chain, nullptr, in_dev, &sc, &desc, &a);
  if (s != MG_OK) return s;
  MG_CUDA(c, launch_pass_yz<T>(sc->n, sc->C, 2, a, c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  return MG_OK;
}

// ---------------------------------------------------------------------------
// Differentiation: K fixed-P sweeps from the chain's current state with the
// noise of its next K sweeps, the loss L = sum_j w_j |s_hat_K,j|^2, and the
// adjoint sweeps back to the start (per-sweep checkpoints of the state).  The
// chain's state, P and sweep counter are restored afterwards.
// ---------------------------------------------------------------------------

template <typename T>
mg_status adjoint_impl(mg_ctx* c, int chain, int K, const double* logP, const double* wl_host, double* loss_out,
                       double* dlogP, double* dd_out) {
  using V2 = typename VT<T>::c2;
  Chain& ch = c->chains[chain];
  const Group& g = c->groups[ch.group];
  const int n = g.n, H = n / 2, B1 = g.B + 1;
  const size_t Mh = size_t(n) * n * (H + 1);
  const size_t main_b = size_t(n) * n * H * sizeof(V2), nyq_b = size_t(n) * n * sizeof(V2);
  const size_t state_b = main_b + nyq_b;
  // the chain's size class, its descriptor and launch arguments
  SizeClass* sc;
  size_t ci;
  if (!find_chain(c, chain, &sc, &ci)) return fail(c, MG_EINVAL, "chain index out of range");
  const ChainDev<T> cd0 = reinterpret_cast<const ChainDev<T>*>(sc->h_desc.data())[ci];
  LaunchArgs<T> base = one_chain_args<T>(*sc, ci, static_cast<const ChainDev<T>*>(sc->d_desc->p) + ci);

  // work buffers, kept between calls for this grid size
  AdjWork& w = c->adj_work[n];
  cudaError_t e;
  if (!w.scr) {
    w.scr = dalloc(state_b, &e);
    MG_CUDA(c, e);
    w.adj = dalloc(state_b, &e);
    MG_CUDA(c, e);
    w.wl64 = dalloc(Mh * sizeof(double), &e);
    MG_CUDA(c, e);
    w.wl = dalloc(Mh * sizeof(T), &e);
    MG_CUDA(c, e);
    w.dd = dalloc(g.M * sizeof(T), &e);
    MG_CUDA(c, e);
    w.ddw = dalloc(g.M * sizeof(double), &e);
    MG_CUDA(c, e);
    w.desc = dalloc(5 * sizeof(ChainDev<T>), &e);
    MG_CUDA(c, e);
    w.sw = dalloc(sizeof(uint32_t), &e);
    MG_CUDA(c, e);
    MG_CUDA(c, cudaStreamCreateWithFlags(&w.up, cudaStreamNonBlocking));
    MG_CUDA(c, cudaEventCreateWithFlags(&w.up_ev, cudaEventDisableTiming));
    LaunchArgs<T> none;  // set the adjoint kernels' attributes (outside any capture)
    std::memset(&none, 0, sizeof(none));
    MG_CUDA(c, launch_pass_yz<T>(n, sc->C, 3, none, c->stream));
    MG_CUDA(c, launch_pass_x<T>(n, 1, none, sc->B_max, c->stream));
    MG_CUDA(c, launch_pass_x<T>(n, 2, none, sc->B_max, c->stream));
  }
  if (!w.acc || w.B1 < B1) {
    w.acc = dalloc(size_t(2) * B1 * sizeof(double), &e);
    MG_CUDA(c, e);
    w.Psave = dalloc(size_t(B1) * sizeof(double), &e);
    MG_CUDA(c, e);
    w.B1 = B1;
  }
  if (w.K_cap < K + 1) {
    w.ck.reset();
    w.ck = dalloc(state_b * size_t(K + 1), &e);
    MG_CUDA(c, e);
    w.K_cap = K + 1;
  }
  char* ckp = static_cast<char*>(w.ck->p);
  auto ck_main = [&](int k) { return reinterpret_cast<V2*>(ckp + size_t(k) * state_b); };
  auto ck_nyq = [&](int k) { return reinterpret_cast<V2*>(ckp + size_t(k) * state_b + main_b); };
  V2* scr_main = static_cast<V2*>(w.scr->p);
  V2* scr_nyq = reinterpret_cast<V2*>(static_cast<char*>(w.scr->p) + main_b);
  V2* adj_main = static_cast<V2*>(w.adj->p);
  V2* adj_nyq = reinterpret_cast<V2*>(static_cast<char*>(w.adj->p) + main_b);
  cudaStream_t s = c->stream;
  uint32_t* ctr = static_cast<uint32_t*>(c->d_sweep->p);
  const uint32_t* sw0 = static_cast<const uint32_t*>(w.sw->p);

  // Small host-to-device uploads first, while the stream holds no kernels (a
  // copy from pageable memory waits for its stream): P = exp(logP) after
  // saving the chain's P, and the four adjoint descriptors:
  //   [0] the chain, [1] pass YZ recomputing t, [2] pass X of the last sweep,
  //   [3] pass X of earlier sweeps, [4] the adjoint pass YZ.
  // The loss weights (n^2 (n/2+1) doubles) go up on a stream of their own
  // once the forward sweeps are queued, so their staging overlaps them.
  MG_CUDA(c, cudaMemcpyAsync(w.Psave->p, ch.P->p, size_t(B1) * sizeof(double), cudaMemcpyDeviceToDevice, s));
  std::vector<double> Pn(B1);
  for (int b = 0; b < B1; ++b) Pn[b] = std::exp(logP[b]);
  MG_CUDA(c, cudaMemcpyAsync(ch.P->p, Pn.data(), size_t(B1) * sizeof(double), cudaMemcpyHostToDevice, s));
  ChainDev<T> dsc[5] = {cd0, cd0, cd0, cd0, cd0};  // [0] unused (the chain's own is in d_desc)
  dsc[1].main = scr_main;
  dsc[1].nyq = scr_nyq;
  for (int k = 2; k <= 3; ++k) {
    dsc[k].main = adj_main;
    dsc[k].nyq = adj_nyq;
    dsc[k].main2 = scr_main;
    dsc[k].nyq2 = scr_nyq;
    dsc[k].wloss = static_cast<const T*>(w.wl->p);
  }
  dsc[2].main_in = ck_main(K);  // the last sweep starts from the final state
  dsc[2].nyq_in = ck_nyq(K);
  dsc[3].main_in = adj_main;  // earlier sweeps transform the adjoint state in place
  dsc[3].nyq_in = adj_nyq;
  dsc[4].main = adj_main;
  dsc[4].nyq = adj_nyq;
  dsc[4].dd = static_cast<T*>(w.dd->p);
  MG_CUDA(c, cudaMemcpyAsync(w.desc->p, dsc, sizeof(dsc), cudaMemcpyHostToDevice, s));
  const ChainDev<T>* dd_ = static_cast<const ChainDev<T>*>(w.desc->p);
  LaunchArgs<T> as = base, ax_top = base, ax_mid = base, ay = base;
  as.chains = dd_ + 1;
  ax_top.chains = dd_ + 2;
  ax_mid.chains = dd_ + 3;
  ay.chains = dd_ + 4;

  // save the chain (state, sweep counter) and draw its coefficients from P
  MG_CUDA(c, cudaMemcpyAsync(w.sw->p, ctr, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  MG_CUDA(c, cudaMemcpyAsync(ck_main(0), ch.main->p, main_b, cudaMemcpyDeviceToDevice, s));
  MG_CUDA(c, cudaMemcpyAsync(ck_nyq(0), ch.nyq->p, nyq_b, cudaMemcpyDeviceToDevice, s));
  mg_status st = launch_shell_draw<T>(c, 0, false);
  if (st != MG_OK) return st;
  MG_CUDA(c, cudaMemsetAsync(w.dd->p, 0, g.M * sizeof(T), s));
  MG_CUDA(c, cudaMemsetAsync(w.acc->p, 0, size_t(2) * B1 * sizeof(double), s));

  // forward: K sweeps of this chain with P fixed, checkpointing every state
  for (int k = 1; k <= K; ++k) {
    sweep_ctr_kernel<<<1, 32, 0, s>>>(ctr, sw0, uint32_t(k - 1));
    MG_CUDA(c, launch_pass_yz<T>(n, sc->C, 0, base, s));
    MG_CUDA(c, launch_pass_x<T>(n, 0, base, sc->B_max, s));
    MG_CUDA(c, cudaMemcpyAsync(ck_main(k), ch.main->p, main_b, cudaMemcpyDeviceToDevice, s));
    MG_CUDA(c, cudaMemcpyAsync(ck_nyq(k), ch.nyq->p, nyq_b, cudaMemcpyDeviceToDevice, s));
  }

  // the loss weights, needed from the first adjoint sweep on
  MG_CUDA(c, cudaMemcpyAsync(w.wl64->p, wl_host, Mh * sizeof(double), cudaMemcpyHostToDevice, w.up));
  adjoint_weights_kernel<T><<<1024, 256, 0, w.up>>>(static_cast<const double*>(w.wl64->p), n,
                                                     static_cast<T*>(w.wl->p));
  MG_CUDA(c, cudaGetLastError());
  MG_CUDA(c, cudaEventRecord(w.up_ev, w.up));
  MG_CUDA(c, cudaStreamWaitEvent(s, w.up_ev, 0));

  // adjoint sweeps K .. 1
  double* grad = static_cast<double*>(w.acc->p);
  for (int k = K; k >= 1; --k) {
    sweep_ctr_kernel<<<1, 32, 0, s>>>(ctr, sw0, uint32_t(k - 1));
    // recompute the forward messenger field of sweep k: y/z transform of t_k
    MG_CUDA(c, cudaMemcpyAsync(scr_main, ck_main(k - 1), main_b, cudaMemcpyDeviceToDevice, s));
    MG_CUDA(c, cudaMemcpyAsync(scr_nyq, ck_nyq(k - 1), nyq_b, cudaMemcpyDeviceToDevice, s));
    MG_CUDA(c, launch_pass_yz<T>(n, sc->C, 0, as, s));
    MG_CUDA(c, launch_pass_x<T>(n, k == K ? 1 : 2, k == K ? ax_top : ax_mid, sc->B_max, s));
    adjoint_reduce_kernel<<<B1, 256, 0, s>>>(cd0.partial, pass_x_tiles(n), B1, grad, grad + B1);
    MG_CUDA(c, cudaGetLastError());
    MG_CUDA(c, launch_pass_yz<T>(n, sc->C, 3, ay, s));
  }
  widen_kernel<T><<<1024, 256, 0, s>>>(static_cast<const T*>(w.dd->p), static_cast<const T*>(g.gamma->p), g.M,
                                        static_cast<double*>(w.ddw->p));
  MG_CUDA(c, cudaGetLastError());
  // restore the chain, then read the results back (the pageable copies wait)
  MG_CUDA(c, cudaMemcpyAsync(ch.main->p, ck_main(0), main_b, cudaMemcpyDeviceToDevice, s));
  MG_CUDA(c, cudaMemcpyAsync(ch.nyq->p, ck_nyq(0), nyq_b, cudaMemcpyDeviceToDevice, s));
  MG_CUDA(c, cudaMemcpyAsync(ch.P->p, w.Psave->p, size_t(B1) * sizeof(double), cudaMemcpyDeviceToDevice, s));
  st = launch_shell_draw<T>(c, 0, false);
  if (st != MG_OK) return st;
  sweep_ctr_kernel<<<1, 32, 0, s>>>(ctr, sw0, 0u);
  MG_CUDA(c, cudaGetLastError());
  std::vector<double> hb(size_t(2) * B1);
  MG_CUDA(c, cudaMemcpyAsync(hb.data(), grad, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  MG_CUDA(c, cudaMemcpyAsync(dd_out, w.ddw->p, g.M * sizeof(double), cudaMemcpyDeviceToHost, s));
  MG_CUDA(c, cudaStreamSynchronize(s));
  double L = 0.0;
  for (int b = 0; b < B1; ++b) {
    dlogP[b] = hb[b];
    L += hb[B1 + b];
  }
  *loss_out = L;
  return MG_OK;
}

mg_status check_status(mg_ctx* c) {
  if (c->sticky != MG_OK) return c->sticky;
  int st = 0;
  MG_CUDA(c, cudaMemcpyAsync(&st, c->d_status->p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (st & kStBounds)
    return fail(c, MG_EBOUNDS, "checked build: a kernel met an index outside its buffer (the access was skipped)");
  if (st & kStTimeout) return fail(c, MG_ETIMEOUT, "a device-side wait ran out of its budget");
  if (st & kStNumeric)
    return fail(c, MG_ENUMERIC, "a shell draw met a non-positive or non-finite sum; the shell kept its P");
  return MG_OK;
}

// Add the current state of every chain to its sums: materialise s into the
// shared scratch field, then add it (the fallback of the fused record mode).
template <typename T>
mg_status accumulate_now(mg_ctx* c) {
  for (size_t ci = 0; ci < c->chains.size(); ++ci) {
    const Group& g = c->groups[c->chains[ci].group];
    T* s = static_cast<T*>(c->d_scratch_s->p);
    Chain& ch = c->chains[ci];
    SizeClass* sc;
    size_t i;
    if (!find_chain(c, int(ci), &sc, &i)) return fail(c, MG_EINVAL, "chain index out of range");
    if (!ch.rec_desc) {  // the chain with the shared scratch field as output, made once
      ChainDev<T> h = reinterpret_cast<const ChainDev<T>*>(sc->h_desc.data())[i];
      h.s_out = s;
      cudaError_t e;
      ch.rec_desc = dalloc(sizeof(h), &e);
      MG_CUDA(c, e);
      MG_CUDA(c, cudaMemcpyAsync(ch.rec_desc->p, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
    }
    const LaunchArgs<T> a = one_chain_args<T>(*sc, i, static_cast<const ChainDev<T>*>(ch.rec_desc->p));
    MG_CUDA(c, launch_pass_yz<T>(sc->n, sc->C, kModeMaterialize, a, c->stream));
    int P, Q;
    split_of(g.n, &P, &Q);
    moments_kernel<T><<<1024, 256, 0, c->stream>>>(s, static_cast<double*>(ch.s1->p), static_cast<double*>(ch.s2->p),
                                                   g.n, P, Q);
    MG_CUDA(c, cudaGetLastError());
  }
  return MG_OK;
}

// Append every chain's P to its trace (the buffer doubles when full).
mg_status append_trace(mg_ctx* c) {
  for (auto& ch : c->chains) {
    const Group& g = c->groups[ch.group];
    const size_t row = size_t(g.B + 1) * sizeof(double);
    if (c->records > ch.trace_cap) {
      const long long cap = std::max<long long>(64, 2 * ch.trace_cap);
      cudaError_t e;
      auto nb = dalloc(size_t(cap) * row, &e);
      MG_CUDA(c, e);
      if (ch.trace && ch.trace_cap > 0)
        MG_CUDA(c, cudaMemcpyAsync(nb->p, ch.trace->p, size_t(ch.trace_cap) * row, cudaMemcpyDeviceToDevice,
                                   c->stream));
      MG_CUDA(c, cudaStreamSynchronize(c->stream));
      ch.trace = nb;
      ch.trace_cap = cap;
    }
    MG_CUDA(c, cudaMemcpyAsync(static_cast<char*>(ch.trace->p) + size_t(c->records - 1) * row, ch.P->p, row,
                               cudaMemcpyDeviceToDevice, c->stream));
  }
  return MG_OK;
}

// After a sweep that ends a record interval: P goes to the trace now; the new
// state goes into the sums inside the next sweep's pass YZ (or now, under the
// persistent schedule).
template <typename T>
mg_status record_sweep(mg_ctx* c) {
  ++c->records;
  mg_status st = append_trace(c);
  if (st != MG_OK) return st;
  if (fused_record(c)) {
    c->stats_pending = true;
    return MG_OK;
  }
  return accumulate_now<T>(c);
}

// A recorded sample still waiting for the next sweep is added now: before
// the sums are read, the state is replaced, or sweeps run that do not record.
mg_status flush_stats(mg_ctx* c) {
  if (!c->stats_pending) return MG_OK;
  const mg_status st = c->precision == 32 ? accumulate_now<float>(c) : accumulate_now<double>(c);
  if (st != MG_OK) return st;
  c->stats_pending = false;
  return MG_OK;
}

mg_status validate_grid(const mg_grid* g) {
  if (!g) return MG_EINVAL;
  if (g->nx != g->ny || g->ny != g->nz) return MG_EUNSUPPORTED;
  if (!(g->L[0] > 0) || g->L[0] != g->L[1] || g->L[1] != g->L[2] || !std::isfinite(g->L[0]))
    return g->L[0] > 0 ? MG_EUNSUPPORTED : MG_EINVAL;
  if (!is_supported_n(g->nx)) return MG_EUNSUPPORTED;
  return MG_OK;
}

template <typename T>
mg_status init_impl(mg_ctx* c, int n_groups, const mg_grid* grids, const double* const* N, const double* const* R,
                    const double* const* d, const double* const* k_edges, const int32_t* n_bins,
                    const uint64_t* seeds, const mg_options* opt) {
  using V2 = typename VT<T>::c2;
  cudaError_t e;
  c->d_sweep = dalloc(2 * sizeof(uint32_t), &e);  // [0] sweep counter, [1] the shell draw's finish ticket
  MG_CUDA(c, e);
  c->d_status = dalloc(sizeof(int), &e);
  MG_CUDA(c, e);
  c->d_rec_now = dalloc(sizeof(int), &e);
  MG_CUDA(c, e);
  MG_CUDA(c, cudaMemsetAsync(c->d_rec_now->p, 0, sizeof(int), c->stream));
  MG_CUDA(c, cudaMemsetAsync(c->d_sweep->p, 0, 2 * sizeof(uint32_t), c->stream));
  MG_CUDA(c, cudaMemsetAsync(c->d_status->p, 0, sizeof(int), c->stream));
  size_t max_M = 0;
  std::map<int, int> class_of_n;
  for (int gi = 0; gi < n_groups; ++gi) {
    const mg_grid& gr = grids[gi];
    Group g;
    g.n = gr.nx;
    g.L = gr.L[0];
    g.B = n_bins[gi];
    g.seed = seeds[gi];
    g.M = size_t(g.n) * g.n * g.n;
    max_M = std::max(max_M, g.M);
    const double* edges = k_edges ? k_edges[gi] : nullptr;
    if (edges) {
      for (int b = 0; b <= g.B; ++b)
        if (!std::isfinite(edges[b]) || (b == 0 ? edges[0] < 0 : edges[b] <= edges[b - 1]))
          return fail(c, MG_EINVAL, "k_edges must be finite, >= 0 and strictly increasing");
    }
    // inputs to the device, tau bound and validation
    auto dN = dalloc(g.M * 8, &e);
    MG_CUDA(c, e);
    auto dR = dalloc(g.M * 8, &e);
    MG_CUDA(c, e);
    auto dd = dalloc(g.M * 8, &e);
    MG_CUDA(c, e);
    auto dmin = dalloc(2 * sizeof(unsigned long long), &e);
    MG_CUDA(c, e);
    MG_CUDA(c, cudaMemcpyAsync(dN->p, N[gi], g.M * 8, cudaMemcpyHostToDevice, c->stream));
    MG_CUDA(c, cudaMemcpyAsync(dR->p, R[gi], g.M * 8, cudaMemcpyHostToDevice, c->stream));
    MG_CUDA(c, cudaMemcpyAsync(dd->p, d[gi], g.M * 8, cudaMemcpyHostToDevice, c->stream));
    unsigned long long init2[2] = {0x7FF0000000000000ull, 0ull};
    MG_CUDA(c, cudaMemcpyAsync(dmin->p, init2, sizeof(init2), cudaMemcpyHostToDevice, c->stream));
    MG_CUDA(c, cudaMemsetAsync(c->d_status->p, 0, sizeof(int), c->stream));
    auto* mb = static_cast<unsigned long long*>(dmin->p);
    tau_bound_kernel<<<1024, 256, 0, c->stream>>>(static_cast<const double*>(dN->p),
                                                  static_cast<const double*>(dR->p),
                                                  static_cast<const double*>(dd->p), g.M, mb, mb + 1,
                                                  static_cast<int*>(c->d_status->p));
    MG_CUDA(c, cudaGetLastError());
    unsigned long long res[2];
    int st = 0;
    MG_CUDA(c, cudaMemcpyAsync(res, dmin->p, sizeof(res), cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(c, cudaMemcpyAsync(&st, c->d_status->p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(c, cudaStreamSynchronize(c->stream));
    if (st & kStBadInput)
      return fail(c, MG_EINVAL, "invalid data: need finite R >= 0, and N > 0 and finite d where R > 0");
    if (res[1] == 0) return fail(c, MG_EINVAL, "no observed voxel (R > 0 nowhere)");
    double bound;
    std::memcpy(&bound, &res[0], sizeof(double));
    g.tau = opt->tau_scale * bound;
    MG_CUDA(c, cudaMemsetAsync(c->d_status->p, 0, sizeof(int), c->stream));
    g.bc = dalloc(g.M * sizeof(V2), &e);
    MG_CUDA(c, e);
    g.gamma = dalloc(g.M * sizeof(T), &e);
    MG_CUDA(c, e);
    messenger_constants_kernel<T><<<1024, 256, 0, c->stream>>>(
        static_cast<const double*>(dN->p), static_cast<const double*>(dR->p), static_cast<const double*>(dd->p), g.M,
        g.tau, static_cast<V2*>(g.bc->p), static_cast<T*>(g.gamma->p));
    MG_CUDA(c, cudaGetLastError());
    // compact row store of the messenger constants (observed z-ranges only)
    {
      // each row's range from R on the device, the offsets (a prefix sum in
      // row order) on the host
      const int n = g.n;
      const size_t rows = size_t(n) * n;
      auto dlohi = dalloc(rows * sizeof(uint32_t), &e);
      MG_CUDA(c, e);
      row_range_kernel<<<1024, 256, 0, c->stream>>>(static_cast<const double*>(dR->p), n, rows,
                                                    static_cast<uint32_t*>(dlohi->p));
      MG_CUDA(c, cudaGetLastError());
      std::vector<uint32_t> lohi(rows);
      MG_CUDA(c, cudaMemcpyAsync(lohi.data(), dlohi->p, rows * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
      MG_CUDA(c, cudaStreamSynchronize(c->stream));
      std::vector<uint32_t> ri(2 * rows);
      uint32_t off = 0;
      for (size_t row = 0; row < rows; ++row) {
        ri[2 * row] = off;
        ri[2 * row + 1] = lohi[row];
        off += (lohi[row] >> 16) - (lohi[row] & 0xffffu);
      }
      g.row_info = dalloc(ri.size() * sizeof(uint32_t), &e);
      MG_CUDA(c, e);
      MG_CUDA(c, cudaMemcpyAsync(g.row_info->p, ri.data(), ri.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream));
      g.bc_rows_len = std::max<uint32_t>(off, 4);
      g.bc_rows = dalloc(size_t(g.bc_rows_len) * sizeof(V2), &e);
      MG_CUDA(c, e);
      pack_rows_kernel<T><<<1024, 256, 0, c->stream>>>(static_cast<const V2*>(g.bc->p),
                                                       static_cast<const uint2*>(g.row_info->p), n,
                                                       static_cast<V2*>(g.bc_rows->p));
      MG_CUDA(c, cudaGetLastError());
    }
    // shells
    const auto tab = build_bin_table(g.n, g.L, g.B, edges, &g.n_b);
    g.bin_of_m2 = dalloc(tab.size(), &e);
    MG_CUDA(c, e);
    MG_CUDA(c, cudaMemcpyAsync(g.bin_of_m2->p, tab.data(), tab.size(), cudaMemcpyHostToDevice, c->stream));
    g.n_b_dev = dalloc(g.n_b.size() * sizeof(long long), &e);
    MG_CUDA(c, e);
    MG_CUDA(c, cudaMemcpyAsync(g.n_b_dev->p, g.n_b.data(), g.n_b.size() * sizeof(long long), cudaMemcpyHostToDevice, c->stream));
    MG_CUDA(c, cudaStreamSynchronize(c->stream));  // dN, dR, dd freed below
    c->B_max = std::max(c->B_max, g.B);
    c->groups.push_back(std::move(g));
    const Group& gg = c->groups.back();
    // chains
    if (!class_of_n.count(gg.n)) {
      class_of_n[gg.n] = int(c->classes.size());
      SizeClass sc;
      sc.n = gg.n;
      int choices[4];
      const int nch = yz_cluster_choices(gg.n, c->precision, choices, 4);
      sc.C = choices[0];
      if (opt->yz_cluster) {
        bool ok = false;
        for (int k = 0; k < nch; ++k) ok = ok || choices[k] == opt->yz_cluster;
        if (!ok) return fail(c, MG_EUNSUPPORTED, "yz_cluster not built for this grid size and precision");
        sc.C = opt->yz_cluster;
      }
      c->classes.push_back(sc);
    }
    SizeClass& sc = c->classes[class_of_n[gg.n]];
    sc.B_max = std::max(sc.B_max, gg.B);
    const int H = gg.n / 2;
    for (int k = 0; k < opt->n_chains; ++k) {
      Chain ch;
      ch.group = gi;
      ch.chain_id = uint32_t(opt->chain_id0 + k);
      const size_t main_b = size_t(gg.n) * gg.n * H * sizeof(V2), nyq_b = size_t(gg.n) * gg.n * sizeof(V2);
      ch.main = dalloc(main_b, &e);
      MG_CUDA(c, e);
      ch.nyq = dalloc(nyq_b, &e);
      MG_CUDA(c, e);
      MG_CUDA(c, cudaMemsetAsync(ch.main->p, 0, main_b, c->stream));
      MG_CUDA(c, cudaMemsetAsync(ch.nyq->p, 0, nyq_b, c->stream));
      ch.coef = dalloc(size_t(gg.B + 2) * sizeof(V2), &e);
      MG_CUDA(c, e);
      ch.mscale = dalloc(size_t(gg.B + 2) * sizeof(T), &e);
      MG_CUDA(c, e);
      MG_CUDA(c, cudaMemsetAsync(ch.mscale->p, 0, size_t(gg.B + 2) * sizeof(T), c->stream));
      ch.partial = dalloc(size_t(pass_x_tiles(gg.n)) * (gg.B + 1) * 2 * sizeof(double), &e);
      MG_CUDA(c, e);
      ch.P = dalloc(size_t(gg.B + 1) * sizeof(double), &e);
      MG_CUDA(c, e);
      ch.sig = dalloc(size_t(gg.B + 1) * sizeof(double), &e);
      MG_CUDA(c, e);
      ch.chi = dalloc(size_t(gg.B + 1) * sizeof(double), &e);
      MG_CUDA(c, e);
      MG_CUDA(c, cudaMemsetAsync(ch.sig->p, 0, size_t(gg.B + 1) * sizeof(double), c->stream));
      MG_CUDA(c, cudaMemsetAsync(ch.chi->p, 0, size_t(gg.B + 1) * sizeof(double), c->stream));
      std::vector<double> P0(gg.B + 1, (gg.L * gg.L * gg.L) / double(gg.M));
      if (opt->P0)
        for (int b = 0; b <= gg.B; ++b) P0[b] = opt->P0[b];
      MG_CUDA(c, cudaMemcpyAsync(ch.P->p, P0.data(), P0.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      if (opt->start_dispersion > 0.0) {
        disperse_start_kernel<<<1, 256, 0, c->stream>>>(static_cast<double*>(ch.P->p), gg.B + 1,
                                                        opt->start_dispersion, uint32_t(gg.seed & 0xffffffffu),
                                                        uint32_t(gg.seed >> 32), ch.chain_id);
        MG_CUDA(c, cudaGetLastError());
      }
      if (c->record_every > 0) {
        ch.s1 = dalloc(gg.M * sizeof(double), &e);
        MG_CUDA(c, e);
        ch.s2 = dalloc(gg.M * sizeof(double), &e);
        MG_CUDA(c, e);
        MG_CUDA(c, cudaMemsetAsync(ch.s1->p, 0, gg.M * sizeof(double), c->stream));
        MG_CUDA(c, cudaMemsetAsync(ch.s2->p, 0, gg.M * sizeof(double), c->stream));
      }
      c->classes[class_of_n[gg.n]].chains.push_back(int(c->chains.size()));
      c->chains.push_back(std::move(ch));
    }
  }
  if (c->record_every > 0) {
    c->d_scratch_s = dalloc(max_M * sizeof(T), &e);
    MG_CUDA(c, e);
  }
  mg_status s = upload_descriptors<T>(c);
  if (s != MG_OK) return s;
  for (auto& sc : c->classes) {
    LaunchArgs<T> none;
    std::memset(&none, 0, sizeof(none));  // n_chains = 0: set kernel attributes only
    for (int mode = 0; mode < 3; ++mode) MG_CUDA(c, launch_pass_yz<T>(sc.n, sc.C, mode, none, c->stream));
    MG_CUDA(c, launch_pass_x<T>(sc.n, 0, none, sc.B_max, c->stream));
    if (c->mixing) {
      MG_CUDA(c, launch_pass_x<T>(sc.n, kXMixDraw, none, sc.B_max, c->stream));
      MG_CUDA(c, launch_pass_x<T>(sc.n, kXMixScale, none, sc.B_max, c->stream));
    }
  }
  s = launch_shell_draw<T>(c, 0, false);
  if (s != MG_OK) return s;
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (opt->persistent) {
    if (!persist_eligible(c))
      return fail(c, MG_EUNSUPPORTED,
                  "persistent launch needs grid sizes 16..128 without y/z clusters, <= 6 sizes, <= 64 chains each");
    if ((s = build_persist<T>(c)) != MG_OK) return s;
    c->persist = true;
  }
  if (opt->autotune && (s = tune_impl<T>(c, 5)) != MG_OK) return s;
  return MG_OK;
}

mg_status create(mg_ctx** out, int32_t n_groups, const mg_grid* grids, const double* const* N,
                 const double* const* R, const double* const* d, const double* const* k_edges,
                 const int32_t* n_bins, const uint64_t* seeds, const mg_options* opt_in) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  if (n_groups < 1 || !grids || !N || !R || !d || !n_bins || !seeds)
    return fail(nullptr, MG_EINVAL, "null argument or n_groups < 1");
  mg_options opt;
  mg_options_init(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.precision != 32 && opt.precision != 64) return fail(nullptr, MG_EINVAL, "precision must be 32 or 64");
  if (opt.n_chains < 1 || opt.chain_id0 < 0) return fail(nullptr, MG_EINVAL, "n_chains >= 1, chain_id0 >= 0");
  if (!(opt.tau_scale > 0.0 && opt.tau_scale <= 1.0)) return fail(nullptr, MG_EINVAL, "tau_scale in (0, 1]");
  if (opt.record_every < 0) return fail(nullptr, MG_EINVAL, "record_every >= 0");
  if (opt.yz_cluster < 0) return fail(nullptr, MG_EINVAL, "yz_cluster >= 0");
  if (opt.mixing < 0 || opt.mixing > 2) return fail(nullptr, MG_EINVAL, "mixing must be 0, 1 or 2");
  if (!(opt.start_dispersion >= 0.0) || !std::isfinite(opt.start_dispersion))
    return fail(nullptr, MG_EINVAL, "start_dispersion must be finite and >= 0");
  if (opt.mixing && opt.fix_P) return fail(nullptr, MG_EINVAL, "mixing sweeps draw P; fix_P must be 0");
  if (opt.mixing && opt.persistent)
    return fail(nullptr, MG_EUNSUPPORTED, "mixing sweeps run one launch per pass (persistent must be 0)");
  for (int g = 0; g < n_groups; ++g) {
    mg_status s = validate_grid(&grids[g]);
    if (s != MG_OK) return fail(nullptr, s, "grid must be cubic with equal sides and n in {8,12,16,24,32,48,64,96,128,192,256}");
    if (n_bins[g] < 1 || n_bins[g] > kMaxBins) return fail(nullptr, MG_EINVAL, "1 <= n_bins <= 254");
    if (!N[g] || !R[g] || !d[g]) return fail(nullptr, MG_EINVAL, "null data array");
    if (opt.P0)
      for (int b = 0; b <= n_bins[g]; ++b)
        if (!(opt.P0[b] > 0.0) || !std::isfinite(opt.P0[b])) return fail(nullptr, MG_EINVAL, "P0 must be positive and finite");
  }
  if (opt.P0) {
    for (int g = 1; g < n_groups; ++g)
      if (n_bins[g] != n_bins[0]) return fail(nullptr, MG_EINVAL, "P0 needs equal n_bins in all groups");
  }
  auto* c = new mg_ctx();
  c->precision = opt.precision;
  c->fix_P = opt.fix_P ? 1 : 0;
  c->mixing = opt.mixing;
  c->record_every = opt.record_every;
  c->timeout = opt.timeout_cycles > 0 ? opt.timeout_cycles : 4000000000ll;
  if (opt.cuda_stream) {
    c->stream = static_cast<cudaStream_t>(opt.cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return MG_ECUDA;
    }
    c->own_stream = true;
  }
  const mg_status s = c->precision == 32
                          ? init_impl<float>(c, n_groups, grids, N, R, d, k_edges, n_bins, seeds, &opt)
                          : init_impl<double>(c, n_groups, grids, N, R, d, k_edges, n_bins, seeds, &opt);
  if (s != MG_OK) {
    mg_destroy(c);
    return s;
  }
  *out = c;
  return MG_OK;
}

bool valid_chain(const mg_ctx* c, int32_t chain) { return chain >= 0 && size_t(chain) < c->chains.size(); }

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

namespace mg {
bool supported_n(int n) { return is_supported_n(n); }
void set_thread_error(const char* msg) { g_create_error = msg; }

int yz_cluster_choices(int n, int precision, int* out, int max_out) {
  std::vector<int> v;
  if (precision == 32) {
    if (n == 256) v = {4, 2, 8};
    else if (n == 192) v = {1, 2};
    else if (n == 128) v = {1, 2};
    else v = {1};
  } else {
    if (n == 256) v = {4};
    else if (n == 192) v = {2};
    else v = {1};
  }
  int k = 0;
  for (int c : v)
    if (k < max_out) out[k++] = c;
  return k;
}
}  // namespace mg

extern "C" {

void mg_options_init(mg_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = 64;
  o->n_chains = 1;
  o->chain_id0 = 0;
  o->tau_scale = 1.0;
  o->P0 = nullptr;
  o->record_every = 0;
  o->fix_P = 0;
  o->timeout_cycles = 0;
  o->cuda_stream = nullptr;
  o->yz_cluster = 0;
  o->persistent = 0;
  o->autotune = 0;
  o->mixing = 0;
  o->start_dispersion = 0.0;
}

mg_status mg_init(mg_ctx** out, const mg_grid* grid, const double* N, const double* R, const double* d,
                  const double* k_edges, int32_t n_bins, uint64_t seed, const mg_options* opt) {
  const double* Np[1] = {N};
  const double* Rp[1] = {R};
  const double* dp[1] = {d};
  const double* ep[1] = {k_edges};
  return create(out, 1, grid, Np, Rp, dp, ep, &n_bins, &seed, opt);
}

mg_status mg_init_batch(mg_ctx** out, int32_t n_groups, const mg_grid* grids, const double* const* N,
                        const double* const* R, const double* const* d, const double* const* k_edges,
                        const int32_t* n_bins, const uint64_t* seeds, const mg_options* opt) {
  return create(out, n_groups, grids, N, R, d, k_edges, n_bins, seeds, opt);
}

mg_status mg_sweep(mg_ctx* c, int64_t n) {
  if (!c) return MG_EINVAL;
  if (c->sticky != MG_OK) return c->sticky;
  if (n < 0) return fail(c, MG_EINVAL, "n_sweeps must be >= 0");
  for (int64_t i = 0; i < n; ++i) {
    mg_status s = MG_OK;
    const bool mix = mixing_sweep_next(c);
    const bool fused = fused_record(c);
    // the record mode of pass YZ adds its incoming state to the sums iff it
    // is a recorded sample not yet added
    if (fused) MG_CUDA(c, cudaMemsetAsync(c->d_rec_now->p, c->stats_pending ? 1 : 0, sizeof(int), c->stream));
    cudaGraphExec_t& graph = mix ? c->graph_mix : c->graph;
    if (!graph && !c->graph_failed) {
      cudaGraph_t g;
      if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        s = enqueue_sweep(c, mix);
        const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (s == MG_OK && e == cudaSuccess) {
          if (cudaGraphInstantiate(&graph, g, 0) != cudaSuccess) {
            graph = nullptr;
            c->graph_failed = true;
          }
          cudaGraphDestroy(g);
        } else {
          c->graph_failed = true;
          (void)cudaGetLastError();
          if (s != MG_OK) return s;
        }
      } else {
        c->graph_failed = true;
        (void)cudaGetLastError();
      }
    }
    if (graph) {
      MG_CUDA(c, cudaGraphLaunch(graph, c->stream));
    } else {
      s = enqueue_sweep(c, mix);
      if (s != MG_OK) return s;
    }
    if (fused) c->stats_pending = false;
    ++c->sweeps;
    if (c->record_every > 0 && c->sweeps % c->record_every == 0) {
      s = c->precision == 32 ? record_sweep<float>(c) : record_sweep<double>(c);
      if (s != MG_OK) return s;
    }
  }
  return MG_OK;
}

mg_status mg_sweep_timed(mg_ctx* c, int64_t n, double* ms_out) {
  if (!c || !ms_out) return MG_EINVAL;
  if (c->sticky != MG_OK) return c->sticky;
  if (n < 0) return fail(c, MG_EINVAL, "n_sweeps must be >= 0");
  // timed sweeps record nothing: a pending sample is added first
  mg_status fs = flush_stats(c);
  if (fs != MG_OK) return fs;
  if (c->d_rec_now) MG_CUDA(c, cudaMemsetAsync(c->d_rec_now->p, 0, sizeof(int), c->stream));
  cudaEvent_t ev[4];
  for (auto& e : ev) MG_CUDA(c, cudaEventCreate(&e));
  for (int64_t i = 0; i < n; ++i) {
    const bool mix = mixing_sweep_next(c);
    MG_CUDA(c, cudaEventRecord(ev[0], c->stream));
    mg_status s = c->precision == 32 ? enqueue_passes<float>(c, 1, mix) : enqueue_passes<double>(c, 1, mix);
    if (s != MG_OK) return s;
    MG_CUDA(c, cudaEventRecord(ev[1], c->stream));
    s = c->precision == 32 ? enqueue_passes<float>(c, 2, mix) : enqueue_passes<double>(c, 2, mix);
    if (s != MG_OK) return s;
    MG_CUDA(c, cudaEventRecord(ev[2], c->stream));
    s = c->precision == 32 ? enqueue_passes<float>(c, 4, mix) : enqueue_passes<double>(c, 4, mix);
    if (s != MG_OK) return s;
    MG_CUDA(c, cudaEventRecord(ev[3], c->stream));
    MG_CUDA(c, cudaEventSynchronize(ev[3]));
    for (int k = 0; k < 3; ++k) {
      float ms = 0.f;
      MG_CUDA(c, cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
      ms_out[k] += double(ms);
    }
    ++c->sweeps;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return check_status(c);
}

mg_status mg_read_s(mg_ctx* c, int32_t chain, void* out, int32_t out_is_device) {
  if (!c || !out) return MG_EINVAL;
  if (c->sticky != MG_OK) return c->sticky;
  if (!valid_chain(c, chain)) return fail(c, MG_EINVAL, "chain index out of range");
  const Group& g = c->groups[c->chains[chain].group];
  const size_t es = c->precision == 32 ? 4 : 8;
  void* dst = out;
  std::shared_ptr<DevBuf> tmp;
  if (!out_is_device) {
    cudaError_t e;
    tmp = dalloc(g.M * es, &e);
    MG_CUDA(c, e);
    dst = tmp->p;
  }
  const mg_status s = c->precision == 32 ? materialize<float>(c, chain, static_cast<float*>(dst))
                                         : materialize<double>(c, chain, static_cast<double*>(dst));
  if (s != MG_OK) return s;
  if (!out_is_device) {
    MG_CUDA(c, cudaMemcpyAsync(out, dst, g.M * es, cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return check_status(c);
}

mg_status mg_read_pk(mg_ctx* c, int32_t chain, double* out) {
  if (!c || !out) return MG_EINVAL;
  if (!valid_chain(c, chain)) return fail(c, MG_EINVAL, "chain index out of range");
  const Group& g = c->groups[c->chains[chain].group];
  MG_CUDA(c, cudaMemcpyAsync(out, c->chains[chain].P->p, size_t(g.B + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_status(c);
}

mg_status mg_read_pk_all(mg_ctx* c, double* out) {
  if (!c || !out) return MG_EINVAL;
  const int B1 = c->B_max + 1;
  const size_t bytes = c->chains.size() * size_t(B1) * sizeof(double);
  if (!c->d_pk_all) {
    cudaError_t e;
    c->d_pk_all = dalloc(bytes, &e);
    MG_CUDA(c, e);
  }
  gather_pk_kernel<<<unsigned(c->chains.size()), 128, 0, c->stream>>>(static_cast<const DrawDev*>(c->d_draw->p), B1,
                                                                     static_cast<double*>(c->d_pk_all->p));
  MG_CUDA(c, cudaGetLastError());
  MG_CUDA(c, cudaMemcpyAsync(out, c->d_pk_all->p, bytes, cudaMemcpyDeviceToHost, c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_status(c);
}

mg_status mg_read_stats(mg_ctx* c, int32_t chain, mg_stats* out) {
  if (!c || !out) return MG_EINVAL;
  if (!valid_chain(c, chain)) return fail(c, MG_EINVAL, "chain index out of range");
  const Chain& ch = c->chains[chain];
  const Group& g = c->groups[ch.group];
  out->sweeps = c->sweeps;
  out->records = c->records;
  out->tau = g.tau;
  out->n_bins = g.B;
  if (out->n_b) std::memcpy(out->n_b, g.n_b.data(), g.n_b.size() * sizeof(long long));
  const size_t nb = size_t(g.B + 1) * sizeof(double);
  if (out->sigma_b) MG_CUDA(c, cudaMemcpyAsync(out->sigma_b, ch.sig->p, nb, cudaMemcpyDeviceToHost, c->stream));
  if (out->chi_b) MG_CUDA(c, cudaMemcpyAsync(out->chi_b, ch.chi->p, nb, cudaMemcpyDeviceToHost, c->stream));
  std::vector<double> s1;
  if (out->mean || out->var) {
    if (c->record_every <= 0) return fail(c, MG_ESTATE, "mean/var need record_every > 0");
    const mg_status fs = flush_stats(c);
    if (fs != MG_OK) return fs;
    s1.resize(g.M);
    MG_CUDA(c, cudaMemcpyAsync(s1.data(), ch.s1->p, g.M * 8, cudaMemcpyDeviceToHost, c->stream));
    if (out->var) MG_CUDA(c, cudaMemcpyAsync(out->var, ch.s2->p, g.M * 8, cudaMemcpyDeviceToHost, c->stream));
  }
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (!s1.empty() && c->precision == 32) {
    // FP32 chains keep each sum as a (hi, lo) pair of floats
    auto widen = [](double* v, size_t n) {
      for (size_t i = 0; i < n; ++i) {
        float hl[2];
        std::memcpy(hl, v + i, sizeof(hl));
        v[i] = double(hl[0]) + double(hl[1]);
      }
    };
    widen(s1.data(), g.M);
    if (out->var) widen(out->var, g.M);
  }
  if (!s1.empty()) {
    // mean = S1 / n, var = (S2 - S1 mean) / (n - 1) over the n recorded
    // samples, from the sums' row-slot order (sums_index) to [x][y][z]
    std::vector<double> s2;
    if (out->var) s2.assign(out->var, out->var + g.M);
    const double n_rec = double(c->records);
    const double inv_n = c->records > 0 ? 1.0 / n_rec : 0.0;
    const double inv_n1 = c->records > 1 ? 1.0 / (n_rec - 1.0) : 0.0;
    int P, Q;
    split_of(g.n, &P, &Q);
    size_t i = 0;
    for (int x = 0; x < g.n; ++x)
      for (int y = 0; y < g.n; ++y)
        for (int z = 0; z < g.n; ++z, ++i) {
          const size_t j = sums_index(g.n, P, Q, x, y, z);
          const double mu = s1[j] * inv_n;
          if (out->mean) out->mean[i] = mu;
          if (out->var) out->var[i] = std::max(0.0, (s2[j] - s1[j] * mu) * inv_n1);
        }
  }
  return check_status(c);
}

mg_status mg_set_s(mg_ctx* c, int32_t chain, const void* s_in, int32_t s_is_device) {
  if (!c || !s_in) return MG_EINVAL;
  if (c->sticky != MG_OK) return c->sticky;
  if (!valid_chain(c, chain)) return fail(c, MG_EINVAL, "chain index out of range");
  const Group& g = c->groups[c->chains[chain].group];
  const size_t es = c->precision == 32 ? 4 : 8;
  {
    const mg_status fs = flush_stats(c);  // a pending sample is the state about to be replaced
    if (fs != MG_OK) return fs;
  }
  const void* src = s_in;
  std::shared_ptr<DevBuf> tmp;
  if (!s_is_device) {
    cudaError_t e;
    tmp = dalloc(g.M * es, &e);
    MG_CUDA(c, e);
    MG_CUDA(c, cudaMemcpyAsync(tmp->p, s_in, g.M * es, cudaMemcpyHostToDevice, c->stream));
    src = tmp->p;
  }
  const mg_status s = c->precision == 32 ? load_s<float>(c, chain, static_cast<const float*>(src))
                                         : load_s<double>(c, chain, static_cast<const double*>(src));
  if (s != MG_OK) return s;
  return check_status(c);
}

mg_status mg_set_pk(mg_ctx* c, int32_t chain, const double* P) {
  if (!c || !P) return MG_EINVAL;
  if (c->sticky != MG_OK) return c->sticky;
  if (!valid_chain(c, chain)) return fail(c, MG_EINVAL, "chain index out of range");
  const Group& g = c->groups[c->chains[chain].group];
  for (int b = 0; b <= g.B; ++b)
    if (!(P[b] > 0.0) || !std::isfinite(P[b])) return fail(c, MG_EINVAL, "P must be positive and finite");
  MG_CUDA(c, cudaMemcpyAsync(c->chains[chain].P->p, P, size_t(g.B + 1) * sizeof(double), cudaMemcpyHostToDevice,
                             c->stream));
  const mg_status s = c->precision == 32 ? launch_shell_draw<float>(c, 0, false) : launch_shell_draw<double>(c, 0, false);
  if (s != MG_OK) return s;
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_status(c);
}

mg_status mg_set_data(mg_ctx* c, int32_t group, const double* d) {
  if (!c || !d) return MG_EINVAL;
  if (c->sticky != MG_OK) return c->sticky;
  if (group < 0 || size_t(group) >= c->groups.size()) return fail(c, MG_EINVAL, "group index out of range");
  const Group& g = c->groups[group];
  for (size_t i = 0; i < g.M; ++i)
    if (!std::isfinite(d[i])) return fail(c, MG_EINVAL, "d must be finite");
  cudaError_t e;
  auto dd = dalloc(g.M * sizeof(double), &e);
  MG_CUDA(c, e);
  MG_CUDA(c, cudaMemcpyAsync(dd->p, d, g.M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (c->precision == 32) {
    set_data_kernel<float><<<1024, 256, 0, c->stream>>>(static_cast<const float*>(g.gamma->p),
                                                        static_cast<const double*>(dd->p), g.M,
                                                        static_cast<float2*>(g.bc->p));
    pack_rows_kernel<float><<<1024, 256, 0, c->stream>>>(static_cast<const float2*>(g.bc->p),
                                                         static_cast<const uint2*>(g.row_info->p), g.n,
                                                         static_cast<float2*>(g.bc_rows->p));
  } else {
    set_data_kernel<double><<<1024, 256, 0, c->stream>>>(static_cast<const double*>(g.gamma->p),
                                                         static_cast<const double*>(dd->p), g.M,
                                                         static_cast<double2*>(g.bc->p));
    pack_rows_kernel<double><<<1024, 256, 0, c->stream>>>(static_cast<const double2*>(g.bc->p),
                                                          static_cast<const uint2*>(g.row_info->p), g.n,
                                                          static_cast<double2*>(g.bc_rows->p));
  }
  MG_CUDA(c, cudaGetLastError());
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_status(c);
}

mg_status mg_adjoint(mg_ctx* c, int32_t chain, int32_t K, const double* logP, const double* w, double* loss,
                     double* dlogP, double* dd) {
  if (!c || !logP || !w || !loss || !dlogP || !dd) return MG_EINVAL;
  if (c->sticky != MG_OK) return c->sticky;
  if (!valid_chain(c, chain)) return fail(c, MG_EINVAL, "chain index out of range");
  if (K < 1) return fail(c, MG_EINVAL, "K must be >= 1");
  const Group& g = c->groups[c->chains[chain].group];
  // the adjoint x pass holds two pencil tiles in shared memory
  if (c->precision == 64 && g.n > 192)
    return fail(c, MG_EUNSUPPORTED, "the FP64 adjoint is built for n <= 192");
  for (int b = 0; b <= g.B; ++b)
    if (!std::isfinite(logP[b])) return fail(c, MG_EINVAL, "logP must be finite");
  const mg_status s = c->precision == 32 ? adjoint_impl<float>(c, chain, K, logP, w, loss, dlogP, dd)
                                         : adjoint_impl<double>(c, chain, K, logP, w, loss, dlogP, dd);
  if (s != MG_OK) return s;
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_status(c);
}

mg_status mg_tune(mg_ctx* c, int32_t reps) {
  if (!c) return MG_EINVAL;
  if (c->sticky != MG_OK) return c->sticky;
  return c->precision == 32 ? tune_impl<float>(c, reps) : tune_impl<double>(c, reps);
}

mg_status mg_schedule(mg_ctx* c, int32_t* n_sizes, int32_t* n, int32_t* yz_cluster, int32_t* persistent) {
  if (!c) return MG_EINVAL;
  if (n_sizes) *n_sizes = int32_t(c->classes.size());
  for (size_t k = 0; k < c->classes.size() && k < 8; ++k) {
    if (n) n[k] = c->classes[k].n;
    if (yz_cluster) yz_cluster[k] = c->classes[k].C;
  }
  if (persistent) *persistent = c->persist ? 1 : 0;
  return MG_OK;
}

mg_status mg_get_sweep_count(mg_ctx* c, int64_t* out) {
  if (!c || !out) return MG_EINVAL;
  uint32_t v = 0;
  MG_CUDA(c, cudaMemcpyAsync(&v, c->d_sweep->p, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  *out = int64_t(v);
  return MG_OK;
}

mg_status mg_set_sweep_count(mg_ctx* c, int64_t sweeps) {
  if (!c) return MG_EINVAL;
  if (sweeps < 0 || sweeps > 0xffffffffll) return fail(c, MG_EINVAL, "sweep count out of range");
  const uint32_t v = uint32_t(sweeps);
  MG_CUDA(c, cudaMemcpyAsync(c->d_sweep->p, &v, sizeof(v), cudaMemcpyHostToDevice, c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  c->sweeps = sweeps;
  return MG_OK;
}

mg_status mg_read_pk_trace(mg_ctx* c, int32_t chain, double* out, int64_t max_records, int64_t* n_records) {
  if (!c) return MG_EINVAL;
  if (c->sticky != MG_OK) return c->sticky;
  if (!valid_chain(c, chain)) return fail(c, MG_EINVAL, "chain index out of range");
  if (max_records < 0) return fail(c, MG_EINVAL, "max_records must be >= 0");
  const Chain& ch = c->chains[chain];
  const size_t row = size_t(c->groups[ch.group].B + 1) * sizeof(double);
  const long long n = std::min<long long>(c->records, max_records);
  if (n_records) *n_records = c->records;
  if (n > 0) {
    if (!out) return fail(c, MG_EINVAL, "null output");
    MG_CUDA(c, cudaMemcpyAsync(out, ch.trace->p, size_t(n) * row, cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return MG_OK;
}

mg_status mg_pk_acf(mg_ctx* c, int32_t chain, int32_t max_lag, double* acf, int32_t* n_c) {
  if (!c || !acf || !n_c) return MG_EINVAL;
  if (c->sticky != MG_OK) return c->sticky;
  if (!valid_chain(c, chain)) return fail(c, MG_EINVAL, "chain index out of range");
  if (max_lag < 0 || max_lag >= c->records)
    return fail(c, MG_EINVAL, "need 0 <= max_lag < recorded P(k) samples (record_every > 0)");
  const Chain& ch = c->chains[chain];
  const int B1 = c->groups[ch.group].B + 1;
  cudaError_t e;
  auto da = dalloc(size_t(B1) * (max_lag + 1) * sizeof(double), &e);
  MG_CUDA(c, e);
  auto dn = dalloc(size_t(B1) * sizeof(int), &e);
  MG_CUDA(c, e);
  pk_acf_kernel<<<B1, 256, 0, c->stream>>>(static_cast<const double*>(ch.trace->p), c->records, B1, max_lag,
                                           static_cast<double*>(da->p), static_cast<int*>(dn->p));
  MG_CUDA(c, cudaGetLastError());
  MG_CUDA(c, cudaMemcpyAsync(acf, da->p, size_t(B1) * (max_lag + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
  MG_CUDA(c, cudaMemcpyAsync(n_c, dn->p, size_t(B1) * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  return MG_OK;
}

mg_status mg_pk_quantiles(mg_ctx* c, int32_t chain, int32_t n_q, const double* q, double* out) {
  if (!c || !q || !out) return MG_EINVAL;
  if (c->sticky != MG_OK) return c->sticky;
  if (!valid_chain(c, chain)) return fail(c, MG_EINVAL, "chain index out of range");
  if (n_q < 1 || n_q > 65535) return fail(c, MG_EINVAL, "1 <= n_q <= 65535");
  for (int i = 0; i < n_q; ++i)
    if (!(q[i] >= 0.0 && q[i] <= 1.0)) return fail(c, MG_EINVAL, "quantiles must lie in [0, 1]");
  if (c->records < 1) return fail(c, MG_EINVAL, "no recorded P(k) samples (record_every > 0)");
  const Chain& ch = c->chains[chain];
  const int B1 = c->groups[ch.group].B + 1;
  cudaError_t e;
  auto dq = dalloc(size_t(n_q) * sizeof(double), &e);
  MG_CUDA(c, e);
  auto dout = dalloc(size_t(B1) * n_q * sizeof(double), &e);
  MG_CUDA(c, e);
  MG_CUDA(c, cudaMemcpyAsync(dq->p, q, size_t(n_q) * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  pk_quantile_kernel<<<dim3(unsigned(B1), unsigned(n_q)), 256, 0, c->stream>>>(
      static_cast<const double*>(ch.trace->p), c->records, B1, static_cast<const double*>(dq->p),
      static_cast<double*>(dout->p));
  MG_CUDA(c, cudaGetLastError());
  MG_CUDA(c, cudaMemcpyAsync(out, dout->p, size_t(B1) * n_q * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  return MG_OK;
}

mg_status mg_pk_rhat(mg_ctx* c, int32_t first_chain, int32_t n_chains, int64_t burn, double* rhat) {
  if (!c || !rhat) return MG_EINVAL;
  if (c->sticky != MG_OK) return c->sticky;
  if (n_chains < 2 || n_chains > 256) return fail(c, MG_EINVAL, "2 <= n_chains <= 256");
  if (!valid_chain(c, first_chain) || !valid_chain(c, first_chain + n_chains - 1))
    return fail(c, MG_EINVAL, "chain index out of range");
  if (burn < 0 || c->records - burn < 2) return fail(c, MG_EINVAL, "need at least 2 recorded samples after burn");
  const int B = c->groups[c->chains[first_chain].group].B;
  std::vector<const double*> ptrs(n_chains);
  for (int j = 0; j < n_chains; ++j) {
    const Chain& ch = c->chains[first_chain + j];
    if (c->groups[ch.group].B != B) return fail(c, MG_EINVAL, "chains must have the same shells");
    ptrs[j] = static_cast<const double*>(ch.trace->p);
  }
  cudaError_t e;
  auto dp = dalloc(ptrs.size() * sizeof(double*), &e);
  MG_CUDA(c, e);
  auto dout = dalloc(size_t(B + 1) * sizeof(double), &e);
  MG_CUDA(c, e);
  MG_CUDA(c, cudaMemcpyAsync(dp->p, ptrs.data(), ptrs.size() * sizeof(double*), cudaMemcpyHostToDevice, c->stream));
  pk_rhat_kernel<<<B + 1, 256, 0, c->stream>>>(static_cast<const double* const*>(dp->p), n_chains, c->records, burn,
                                               B + 1, static_cast<double*>(dout->p));
  MG_CUDA(c, cudaGetLastError());
  MG_CUDA(c, cudaMemcpyAsync(rhat, dout->p, size_t(B + 1) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  return MG_OK;
}

mg_status mg_chain_info(mg_ctx* c, int32_t chain, int32_t* n, int32_t* n_bins, int32_t* n_chains) {
  if (!c) return MG_EINVAL;
  if (n_chains) *n_chains = int32_t(c->chains.size());
  if (n || n_bins) {
    if (!valid_chain(c, chain)) return fail(c, MG_EINVAL, "chain index out of range");
    const Group& g = c->groups[c->chains[chain].group];
    if (n) *n = g.n;
    if (n_bins) *n_bins = g.B;
  }
  return MG_OK;
}

mg_status mg_sync(mg_ctx* c) {
  if (!c) return MG_EINVAL;
  MG_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_status(c);
}

mg_status mg_inject_cuda_error(mg_ctx* c, int32_t after_calls) {
  if (!c || after_calls < 0) return MG_EINVAL;
  c->fault_in = after_calls;
  return MG_OK;
}

int32_t mg_build_flags(void) {
#ifdef MG_CHECKED
  return MG_BUILD_CHECKED;
#else
  return 0;
#endif
}

const char* mg_last_error(const mg_ctx* c) {
  if (!c) return g_create_error.empty() ? "null context" : g_create_error.c_str();  // init and no-context calls
  return c->err.c_str();
}

void mg_destroy(mg_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->graph_mix) cudaGraphExecDestroy(c->graph_mix);
  for (cudaStream_t st : c->aux) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (cudaEvent_t ev : c->aux_ev) cudaEventDestroy(ev);
  c->classes.clear();
  c->chains.clear();
  c->groups.clear();
  c->d_draw.reset();
  c->d_pk_all.reset();
  c->adj_work.clear();
  c->d_sweep.reset();
  c->d_status.reset();
  c->d_scratch_s.reset();
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

mg_status mg_normals(int32_t precision, const uint32_t* words_device, int64_t n_pairs, void* out_device,
                     void* stream) {
  if ((precision != 64 && precision != 32) || n_pairs < 0) return MG_EINVAL;
  if (n_pairs == 0) return MG_OK;
  if (!words_device || !out_device) return MG_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = int(std::min<int64_t>((n_pairs + 255) / 256, 4096));
  if (precision == 64)
    normals_kernel<double><<<blocks, 256, 0, st>>>(words_device, (long long)n_pairs, static_cast<double*>(out_device));
  else
    normals_kernel<float><<<blocks, 256, 0, st>>>(words_device, (long long)n_pairs, static_cast<float*>(out_device));
  if (cudaGetLastError() != cudaSuccess) return MG_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MG_ECUDA;
  return MG_OK;
}

mg_status mg_philox(uint64_t seed, uint32_t ctr0, uint32_t ctr1, uint32_t ctr2, uint32_t ctr3, int64_t n_calls,
                    uint32_t* out_device, void* stream) {
  if (n_calls < 0 || (n_calls > 0 && !out_device)) return MG_EINVAL;
  if (n_calls == 0) return MG_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = int(std::min<int64_t>((n_calls + 255) / 256, 4096));
  philox_fill_kernel<<<blocks, 256, 0, st>>>(uint32_t(seed & 0xffffffffu), uint32_t(seed >> 32), ctr0, ctr1, ctr2,
                                              ctr3, (long long)n_calls, reinterpret_cast<uint4*>(out_device));
  if (cudaGetLastError() != cudaSuccess) return MG_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MG_ECUDA;
  return MG_OK;
}

}  // extern "C"
