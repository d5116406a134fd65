// C ABI of libisdf: handle, workspaces and the four steps of the k-ISDF
// fragment-ERI path (Section II of the paper; see include/isdf.h).
//
// Step -> kernels
//   build_points   ao_eval (Eq. 1), ip_init/ip_step (Section II.A), gather_x
//   fit_zeta       G^k = conj(X^k) X^k^T (zgemm), k-convolution |DFT|^2 -> Pi^q
//                  (kdft_cols, Eq. 4 / Algorithm 1); g^k = conj(X^k) Phi^k (zgemm),
//                  k-convolution -> eta^q (Eq. 5); pivoted Cholesky of Pi^q and
//                  W = L_S^{-1} (Eq. 3); xi^q = W eta^q (zeta^q = W^H xi^q).
//   coulomb_metric grid FFT of e^{-iq.r} xi^q with sqrt(4 pi/|q+G|^2) (Eq. 6),
//                  V_xi = Omega c'^* c'^T, V_xi = L_xi L_xi^H, L^q = W^T L_xi so
//                  that V^q = L^q L^q^H = W^T V_xi conj(W).
//   fragment_eri   T^k = X^k C^k, t = DFT_k(T), pair products, DFT_R -> M^q
//                  (Eq. 20 / Algorithm 2); B = [M^q L^q]_q; E = B B^H (Eq. 19);
//                  chemist's permutation and the J/K traces.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "../../include/isdf.h"
#include "common.cuh"

namespace isdf {
thread_local int64_t* g_launch_counter = nullptr;
}

using namespace isdf;

namespace {

constexpr double kTieEps = 1e-11;  // interpolation-point tie window (relative to d_max,0)
constexpr int kIpSplit = 16;       // column-generation split of the (k, mu) sum

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct isdf_handle {
  int device = 0;
  cudaStream_t st = nullptr;
  isdf_precision prec = ISDF_FP64;
  CellDev cell{};
  double volume = 0;
  int nao = 0, nk = 0, ng = 0, np = 0;
  // basis (host copies and device arrays)
  std::vector<int> ao_shell, ao_lxyz, sh_atom, sh_off;
  std::vector<double> prim_exp, prim_norm, coords;
  int maxprim = 1;
  BasisDev bdev{};
  // owned device buffers by name
  std::vector<std::pair<std::string, DevBuf>> bufs;
  bool has_points = false, has_fit = false, has_xi = false, has_eta = false, has_coulomb = false;
  std::vector<int32_t> ips;
  std::vector<int32_t> ranks;    // rank r_q of the truncated factor of Pi^q, per q
  std::vector<int32_t> ranks_v;  // rank n_q of V_xi^q (columns of L^q), per q
  int xi_rows = 0;               // rows of xi kept per q: max_q r_q (rows beyond r_q are zero)
  std::string err;
  int64_t launches = 0;
  std::vector<int2> tiles_host;
  std::vector<int> tile_of_host;
  std::vector<int2> orb_host;
  // device bytes for one q-chunk of the fp16 slices of B (mixed contraction)
  size_t split_budget = (size_t)12 << 30;
  // pair q with -q in the fragment contraction (time-reversal symmetry)
  bool q_sym = true;
  // schedule of the E' contraction's tiles, tuned per size class of the tile list
  // unless fixed by isdf_set_tile_schedule
  bool autotune = true;
  int fixed_cfg = 0, fixed_band = 12;
  struct TuneEntry {
    int bucket;       // floor(log2(tiles))
    int64_t ntiles;   // tile count it was tuned on
    int cfg;          // chosen pipeline of the tile kernel
    int band;         // chosen row blocks per band
    float ms[4];      // first-chunk times of the candidate schedules
  };
  std::vector<TuneEntry> tune_log;
  // per-stage event timing
  static constexpr int kStages = 7;
  bool timing = false;
  double stage_ms[kStages] = {0};
  int64_t stage_n[kStages] = {0};
  double stage_flops[kStages] = {0};
  struct Pending {
    int stage;
    cudaEvent_t a, b;
    double flops;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  cudaEvent_t get_event() {
    if (!event_pool.empty()) {
      cudaEvent_t e = event_pool.back();
      event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // Resolve recorded event pairs (the stream must have been synchronised).
  void resolve_timing() {
    for (auto& p : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        stage_ms[p.stage] += ms;
        stage_n[p.stage] += 1;
        stage_flops[p.stage] += p.flops;
      }
      event_pool.push_back(p.a);
      event_pool.push_back(p.b);
    }
    pending.clear();
  }

  void* buf(const char* name) {
    for (auto& b : bufs)
      if (b.first == name) return b.second.p;
    return nullptr;
  }
  // Ensure a named device buffer of at least `bytes`; returns nullptr on OOM.
  void* ensure(const char* name, size_t bytes) {
    if (bytes == 0) bytes = 16;
    for (auto& b : bufs)
      if (b.first == name) {
        if (b.second.bytes >= bytes) return b.second.p;
        cudaFree(b.second.p);
        b.second.p = nullptr;
        b.second.bytes = 0;
        if (cudaMalloc(&b.second.p, bytes) != cudaSuccess) {
          cudaGetLastError();
          return nullptr;
        }
        b.second.bytes = bytes;
        return b.second.p;
      }
    DevBuf d;
    if (cudaMalloc(&d.p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    d.bytes = bytes;
    bufs.emplace_back(name, d);
    return d.p;
  }
  void release(const char* name) {
    for (auto& b : bufs)
      if (b.first == name && b.second.p) {
        cudaFree(b.second.p);
        b.second.p = nullptr;
        b.second.bytes = 0;
      }
  }
  // Two groups of large buffers never live at once when HBM is short: the
  // grid-sized fit intermediates (eta, xi and their work) and the per-fragment
  // scratch.  An allocation in one group that fails frees the other group and
  // is tried again; freeing the fit group drops eta and xi (a later isdf_get of
  // them, or isdf_coulomb_metric_eta, then needs a new isdf_fit_zeta).
  static bool in_frag_group(const std::string& n) { return n.rfind("frag_", 0) == 0 || n.rfind("tc_", 0) == 0; }
  static bool in_fit_group(const std::string& n) {
    return n == "eta" || n == "xi" || n == "grid_work" || n == "grid_work_emu" || n == "grid_work_v";
  }
  bool evict_other(const char* name) {
    const std::string n(name);
    bool freed = false;
    const bool frag = in_frag_group(n);
    for (auto& b : bufs) {
      const bool other = frag ? in_fit_group(b.first) : in_frag_group(b.first);
      if (other && b.second.p) {
        cudaFree(b.second.p);
        b.second.p = nullptr;
        b.second.bytes = 0;
        freed = true;
      }
    }
    if (freed && frag) has_xi = has_eta = false;
    return freed;
  }
  void* ensure_evict(const char* name, size_t bytes) {
    void* p = ensure(name, bytes);
    if (!p && evict_other(name)) p = ensure(name, bytes);
    return p;
  }
};

namespace {

// Records a CUDA event pair around a block of launches of one stage.
struct StageTimer {
  isdf_handle* h;
  int stage;
  double flops;
  cudaEvent_t a = nullptr;
  StageTimer(isdf_handle* hh, int st, double fl) : h(hh), stage(st), flops(fl) {
    if (h->timing) {
      a = h->get_event();
      cudaEventRecord(a, h->st);
    }
  }
  ~StageTimer() {
    if (h->timing && a) {
      cudaEvent_t b = h->get_event();
      cudaEventRecord(b, h->st);
      h->pending.push_back({stage, a, b, flops});
    }
  }
};

struct LaunchScope {
  int64_t* prev;
  isdf_handle* h;
  explicit LaunchScope(isdf_handle* hh) : prev(g_launch_counter), h(hh) { g_launch_counter = &h->launches; }
  ~LaunchScope() {
    g_launch_counter = prev;
    if (!h->pending.empty() && cudaStreamSynchronize(h->st) == cudaSuccess) h->resolve_timing();
  }
};

int fail(isdf_handle* h, int code, const char* fmt, ...) {
  char b[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b, sizeof(b), fmt, ap);
  va_end(ap);
  if (h) h->err = b;
  return code;
}

#define CK(expr)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(h, ISDF_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),      \
                  __FILE__, __LINE__);                                                             \
  } while (0)

#define ENSURE(var, type, name, count)                                                             \
  type* var = static_cast<type*>(h->ensure_evict(name, sizeof(type) * (size_t)(count)));           \
  if (!var) return fail(h, ISDF_ERR_OOM, "device allocation of %s (%zu bytes) failed", name,      \
                        sizeof(type) * (size_t)(count));

double dfact(int n) {
  double r = 1.0;
  while (n > 1) {
    r *= n;
    n -= 2;
  }
  return r;
}

double prim_norm(double a, int lx, int ly, int lz) {
  const int l = lx + ly + lz;
  const double n2 = std::pow(2.0 * a / M_PI, 1.5) * std::pow(4.0 * a, l) /
                    (dfact(2 * lx - 1) * dfact(2 * ly - 1) * dfact(2 * lz - 1));
  return std::sqrt(n2);
}

// Algorithmic flops of the pair tensor: T = X C, the k->R DFT of T, the pair
// products and the R->q DFT (direct per-axis DFTs: n_a complex MACs per point and axis).
// The q-points whose terms enter E = sum_q B^q B^q^H, with sqrt-weights sw[q].
// With the time-reversal pairing (real AOs on a Gamma-centred mesh give
// V^{-q} = conj(V^q); M^{-q}_{(qp)} = conj(M^q_{(pq)}) holds for any orbitals),
// P_{-q} = swapconj(P_q) for P_q = B^q B^q^H, so E = G + swapconj(G) with
// G = sum_{q in S} w_q P_q over about half the mesh:
//   S = { m_0 in [0, n_0/2], and m_1 in [0, n_1/2] when m_0 is its own negative },
//   w_q = 1/2 when both m_0 and m_1 are their own negatives, else 1,
// which gives every P_q total weight one in G + swapconj(G).  Without the
// pairing S is the whole mesh with unit weights.
void q_point_set(const KMesh& km, bool pair, std::vector<int>& qs, std::vector<double>& sw) {
  const int n0 = km.n[0], n1 = km.n[1], n2 = km.n[2], nk = n0 * n1 * n2;
  qs.clear();
  sw.assign(nk, 1.0);
  for (int q = 0; q < nk; ++q) {
    if (!pair) {
      qs.push_back(q);
      continue;
    }
    const int m0 = q / (n1 * n2), m1 = (q / n2) % n1;
    const bool self0 = (m0 == 0) || (2 * m0 == n0), self1 = (m1 == 0) || (2 * m1 == n1);
    const bool in = (2 * m0 <= n0) && (!self0 || 2 * m1 <= n1);
    if (!in) continue;
    qs.push_back(q);
    if (self0 && self1) sw[q] = std::sqrt(0.5);
  }
}

// Representatives of the pairs {q, -q} (q <= -q in index order, self-conjugate
// q included) in runs of consecutive q, and (dst, src) = (q, -q) for the rest.
// For a real AO basis on a Gamma-centred mesh Pi^{-q} = conj(Pi^q) and
// eta^{-q} = conj(eta^q), so the factor, xi and V_xi of -q are the conjugates
// of those of q.  Without pairing every q is its own representative.
struct QHalf {
  std::vector<std::pair<int, int>> runs;  // (first q, count)
  std::vector<int2> mirror;               // (q, -q) for q not computed
  int count = 0;                          // computed q-points
};
QHalf fit_q_set(const KMesh& km, bool pair) {
  const int n0 = km.n[0], n1 = km.n[1], n2 = km.n[2], nk = n0 * n1 * n2;
  QHalf h;
  for (int q = 0; q < nk; ++q) {
    const int m0 = q / (n1 * n2), m1 = (q / n2) % n1, m2 = q % n2;
    const int mq = (((n0 - m0) % n0) * n1 + (n1 - m1) % n1) * n2 + (n2 - m2) % n2;
    if (pair && mq < q) {
      h.mirror.push_back(make_int2(q, mq));
      continue;
    }
    ++h.count;
    if (!h.runs.empty() && h.runs.back().first + h.runs.back().second == q)
      ++h.runs.back().second;
    else
      h.runs.push_back({q, 1});
  }
  return h;
}

double frag_m_flops(int nk, int np, int nf, int nao, const KMesh& km) {
  const double per_pt = 8.0 * (km.n[0] + km.n[1] + km.n[2]);
  return 8.0 * nk * (double)np * nf * nao + per_pt * nk * (double)np * nf + 6.0 * nk * (double)nf * nf * np +
         per_pt * nk * (double)nf * nf * np;
}

int check_device(isdf_handle* h) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(h, ISDF_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev != h->device)
    return fail(h, ISDF_ERR_STATE, "current device %d differs from the handle's device %d", dev, h->device);
  return ISDF_OK;
}

int upload_basis(isdf_handle* h) {
  auto up = [&](const char* name, const void* src, size_t bytes) -> void* {
    void* d = h->ensure(name, bytes);
    if (!d) return nullptr;
    if (cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
    return d;
  };
  BasisDev& b = h->bdev;
  b.nao = h->nao;
  b.nshell = (int)h->sh_atom.size();
  b.maxprim = h->maxprim;
  b.ao_shell = (const int*)up("ao_shell", h->ao_shell.data(), h->ao_shell.size() * sizeof(int));
  b.ao_lxyz = (const int*)up("ao_lxyz", h->ao_lxyz.data(), h->ao_lxyz.size() * sizeof(int));
  b.sh_atom = (const int*)up("sh_atom", h->sh_atom.data(), h->sh_atom.size() * sizeof(int));
  b.sh_off = (const int*)up("sh_off", h->sh_off.data(), h->sh_off.size() * sizeof(int));
  b.prim_exp = (const double*)up("prim_exp", h->prim_exp.data(), h->prim_exp.size() * sizeof(double));
  b.prim_norm = (const double*)up("prim_norm", h->prim_norm.data(), h->prim_norm.size() * sizeof(double));
  b.coords = (const double*)up("coords", h->coords.data(), h->coords.size() * sizeof(double));
  b.prim_cn = nullptr;
  if (!b.ao_shell || !b.ao_lxyz || !b.sh_atom || !b.sh_off || !b.prim_exp || !b.prim_norm || !b.coords)
    return fail(h, ISDF_ERR_OOM, "uploading the basis failed");
  double2 tw[192];
  grid_twiddles(h->cell.mesh, tw);
  if (!up("grid_tw", tw, sizeof(tw))) return fail(h, ISDF_ERR_OOM, "uploading twiddles failed");
  return ISDF_OK;
}

// Evaluate Phi into the handle (all precisions keep Phi in FP64).
int eval_phi(isdf_handle* h) {
  ENSURE(phi, double2, "phi", (size_t)h->nk * h->nao * h->ng);
  ENSURE(work, double, "ao_work", ao_eval_work_bytes(h->cell, h->bdev) / sizeof(double) + 2);
  CK(ao_eval(h->st, h->cell, h->bdev, phi, work));
  return ISDF_OK;
}

int finish_points(isdf_handle* h) {
  const int np = h->np;
  double2* phi = (double2*)h->buf("phi");
  int32_t* ipsd = (int32_t*)h->buf("ips");
  ENSURE(X, double2, "X", (size_t)h->nk * np * h->nao);
  CK(gather_x(h->st, phi, h->nk, h->nao, h->ng, ipsd, np, X));
  h->has_points = true;
  h->has_fit = h->has_xi = h->has_eta = h->has_coulomb = false;
  return ISDF_OK;
}

}  // namespace

// Groups of fragments for the mixed contraction.  A fragment whose lower
// triangle of 128 x 128 tiles fills kWaves waves of the GPU or more goes alone;
// smaller ones are stacked (ascending size) while the group's scratch -- pair
// rows Z and M^q per row (padded to a tile boundary), and E per fragment -- stays
// within what the largest fragment of the call needs alone (or kMinBytes).
std::vector<std::vector<int>> fragment_groups(int n, const int32_t* n_orb, int nk, int nS, int np, double esz) {
  constexpr int64_t kWaves = 4, kSMs = 152;
  constexpr double kMinBytes = 4.0 * (1 << 30);
  const double per_row = esz * (double)np * (4.0 * nk + 8.0 * nS);
  auto n2of = [&](int f) { return (int64_t)n_orb[f] * n_orb[f]; };
  int64_t n2max = 0;
  for (int f = 0; f < n; ++f) n2max = std::max(n2max, n2of(f));
  const double cap = std::max(kMinBytes, per_row * (double)((n2max + 127) / 128 * 128) +
                                             16.0 * (double)n2max * (double)n2max);
  std::vector<int> order(n);
  for (int f = 0; f < n; ++f) order[f] = f;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n2of(a) < n2of(b); });
  std::vector<std::vector<int>> groups;
  std::vector<int> cur;
  double cur_bytes = 0.0;
  for (int f : order) {
    const int64_t n2 = n2of(f), nt = (n2 + 127) / 128;
    if (nt * (nt + 1) / 2 >= kWaves * kSMs) {
      groups.push_back({f});
      continue;
    }
    const double b = per_row * (double)((n2 + 127) / 128 * 128) + 16.0 * (double)n2 * (double)n2;
    if (!cur.empty() && cur_bytes + b > cap) {
      groups.push_back(cur);
      cur.clear();
      cur_bytes = 0.0;
    }
    cur.push_back(f);
    cur_bytes += b;
  }
  if (!cur.empty()) groups.push_back(cur);
  // largest scratch first, so that the buffers are sized once per call
  std::stable_sort(groups.begin(), groups.end(), [&](const std::vector<int>& a, const std::vector<int>& b) {
    int64_t ra = 0, rb = 0;
    for (int f : a) ra += (n2of(f) + 127) / 128 * 128;
    for (int f : b) rb += (n2of(f) + 127) / 128 * 128;
    return ra > rb;
  });
  return groups;
}

// Schedule of the E' contraction: the pipeline of the tile kernel (cfg 0: K rows of
// 64 fp16 in 3 stages; cfg 1: rows of 32 fp16 in 6 stages) and the band width of
// the tile order (row blocks per band, see syrk_tc_tiles).  Chosen per size class
// of the tile list by timing the first q-chunk with each candidate on first use,
// after one untimed run of each pipeline (the first launch of a kernel pays its
// module loading); the choice is kept in the handle.  `trial(cfg, band)` runs that
// chunk (it overwrites the workspace, so the caller's run of the chunk afterwards
// is unaffected).
struct TileSchedule {
  int cfg, band;
};
constexpr TileSchedule kTileCandidates[4] = {{0, 12}, {1, 12}, {1, 6}, {1, 24}};

TileSchedule tuned_schedule(isdf_handle* h, int64_t ntiles, const std::function<int(int, int)>& trial) {
  const TileSchedule dflt = {h->fixed_cfg, h->fixed_band};
  if (!h->autotune || ntiles < 2 * 152) return dflt;
  const int bucket = (int)std::floor(std::log2((double)ntiles));
  for (const auto& e : h->tune_log)
    if (e.bucket == bucket) return {e.cfg, e.band};
  isdf_handle::TuneEntry t{bucket, ntiles, dflt.cfg, dflt.band, {0, 0, 0, 0}};
  for (int cfg = 0; cfg < 2; ++cfg)
    if (trial(cfg, kTileCandidates[0].band) != 0) return {-1, -1};
  float best = 1e30f;
  for (int i = 0; i < 4; ++i) {
    cudaEvent_t a = h->get_event(), b = h->get_event();
    cudaEventRecord(a, h->st);
    if (trial(kTileCandidates[i].cfg, kTileCandidates[i].band) != 0) return {-1, -1};
    cudaEventRecord(b, h->st);
    if (cudaEventSynchronize(b) != cudaSuccess) return {-1, -1};
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    h->event_pool.push_back(a);
    h->event_pool.push_back(b);
    t.ms[i] = ms;
    if (ms < best) {
      best = ms;
      t.cfg = kTileCandidates[i].cfg;
      t.band = kTileCandidates[i].band;
    }
  }
  h->tune_log.push_back(t);
  return {t.cfg, t.band};
}

// Shared tail of both Coulomb routes: factor V_xi = L_xi L_xi^H, L^q = W^T L_xi
// (so V^q = L^q L^q^H), optional output of V^q, precision copies for the fragments.
int coulomb_tail(isdf_handle* h, double2* Vxi, void* V_out) {
  const int nk = h->nk, np = h->np;
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  double2* W = (double2*)h->buf("W");
  // V_xi = L_xi L_xi^H ; L^q = W^T L_xi
  ENSURE(LtV, double2, "LtV", (size_t)nk * np * np);
  ENSURE(permV, int32_t, "permV", (size_t)nk * np);
  ENSURE(rankV, int32_t, "rankV", nk);
  ENSURE(dwork, double, "chol_dwork", (size_t)nk * 2 * np);
  CK(pchol_batched(h->st, Vxi, np, nk, 1e-15, LtV, permV, rankV, dwork));
  h->ranks_v.assign(nk, 0);
  CK(cudaMemcpyAsync(h->ranks_v.data(), rankV, sizeof(int32_t) * nk, cudaMemcpyDeviceToHost, h->st));
  ENSURE(Lxi, double2, "W_work", (size_t)nk * np * np);
  CK(lt_to_rowmajor(h->st, LtV, rankV, np, nk, Lxi));
  ENSURE(Lq, double2, "Lq", (size_t)nk * np * np);
  CK(zgemm(h->st, 'T', 'N', np, np, np, one, W, np, (int64_t)np * np, Lxi, np, (int64_t)np * np, zero, Lq, np,
           (int64_t)np * np, nk));
  if (V_out) {
    // V^q = W^T V_xi conj(W)
    double2* tmp = Lxi;  // reuse
    CK(zgemm(h->st, 'N', 'R', np, np, np, one, Vxi, np, (int64_t)np * np, W, np, (int64_t)np * np, zero, tmp, np,
             (int64_t)np * np, nk));
    CK(zgemm(h->st, 'T', 'N', np, np, np, one, W, np, (int64_t)np * np, tmp, np, (int64_t)np * np, zero,
             (double2*)V_out, np, (int64_t)np * np, nk));
  }
  if (h->prec == ISDF_MIXED) {
    ENSURE(Xf, float2, "X_f", (size_t)nk * np * h->nao);
    CK(z2c(h->st, (const double2*)h->buf("X"), Xf, (int64_t)nk * np * h->nao));
  }
  CK(cudaStreamSynchronize(h->st));
  h->has_coulomb = true;
  return ISDF_OK;
}

extern "C" {

int isdf_create(const isdf_cell_desc* c, isdf_precision precision, void* cuda_stream, isdf_handle** out) {
  if (!out) return ISDF_ERR_ARG;
  *out = nullptr;
  if (!c) return ISDF_ERR_ARG;
  if (precision != ISDF_FP64 && precision != ISDF_MIXED && precision != ISDF_FP64_TC) return ISDF_ERR_ARG;
  if (c->natm < 1 || c->nshell < 1 || !c->coords || !c->shell_atom || !c->shell_l || !c->shell_nprim ||
      !c->exps || !c->coefs)
    return ISDF_ERR_ARG;
  int64_t nk = 1, ng = 1;
  for (int a = 0; a < 3; ++a) {
    if (c->kmesh[a] < 1 || c->kmesh[a] > 16 || c->mesh[a] < 1 || c->mesh[a] > 64) return ISDF_ERR_ARG;
    nk *= c->kmesh[a];
    ng *= c->mesh[a];
  }
  if (nk > 1024) return ISDF_ERR_ARG;
  isdf_handle* h = new isdf_handle();
  h->prec = precision;
  h->st = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return ISDF_ERR_CUDA;
  }
  // basis
  int nao = 0, poff = 0, maxprim = 1;
  for (int s = 0; s < c->nshell; ++s) {
    const int l = c->shell_l[s], npr = c->shell_nprim[s], at = c->shell_atom[s];
    if (l < 0 || l > 4 || npr < 1 || at < 0 || at >= c->natm) {
      delete h;
      return ISDF_ERR_ARG;
    }
    for (int p = 0; p < npr; ++p)
      if (!(c->exps[poff + p] > 0.0) || !std::isfinite(c->coefs[poff + p])) {
        delete h;
        return ISDF_ERR_ARG;
      }
    maxprim = std::max(maxprim, npr);
    h->sh_atom.push_back(at);
    h->sh_off.push_back(poff);
    for (int p = 0; p < npr; ++p) h->prim_exp.push_back(c->exps[poff + p]);
    poff += npr;
    nao += (l + 1) * (l + 2) / 2;
  }
  h->sh_off.push_back(poff);
  if (nao > 1024) {
    delete h;
    return ISDF_ERR_ARG;
  }
  h->maxprim = maxprim;
  h->prim_norm.assign((size_t)nao * maxprim, 0.0);
  int mu = 0;
  for (int s = 0; s < c->nshell; ++s) {
    const int l = c->shell_l[s];
    for (int lx = l; lx >= 0; --lx)
      for (int ly = l - lx; ly >= 0; --ly) {
        const int lz = l - lx - ly;
        h->ao_shell.push_back(s);
        h->ao_lxyz.push_back(lx);
        h->ao_lxyz.push_back(ly);
        h->ao_lxyz.push_back(lz);
        for (int p = 0; p < c->shell_nprim[s]; ++p) {
          const int gi = h->sh_off[s] + p;
          h->prim_norm[(size_t)mu * maxprim + p] = c->coefs[gi] * prim_norm(c->exps[gi], lx, ly, lz);
        }
        ++mu;
      }
  }
  h->coords.assign(c->coords, c->coords + 3 * c->natm);
  h->nao = nao;
  h->nk = (int)nk;
  h->ng = (int)ng;
  // cell
  CellDev& cd = h->cell;
  std::memcpy(cd.lat, c->lattice, sizeof(cd.lat));
  const double* A = c->lattice;
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (!(std::fabs(det) > 0)) {
    delete h;
    return ISDF_ERR_ARG;
  }
  h->volume = std::fabs(det);
  // rec = 2 pi inv(A)^T : rows b_i
  double inv[9];
  inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  inv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  inv[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  inv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) cd.rec[i * 3 + j] = 2.0 * M_PI * inv[j * 3 + i];
  for (int a = 0; a < 3; ++a) {
    cd.kmesh[a] = c->kmesh[a];
    cd.mesh[a] = c->mesh[a];
  }
  cd.expcut = (c->lattice_eps > 0.0 && c->lattice_eps < 1.0) ? -std::log(c->lattice_eps) : 40.0;
  double amin = 1e300;
  for (double e : h->prim_exp) amin = std::min(amin, e);
  const double rcut = std::sqrt(cd.expcut / amin);
  for (int a = 0; a < 3; ++a) {
    const double bn = std::sqrt(cd.rec[a * 3] * cd.rec[a * 3] + cd.rec[a * 3 + 1] * cd.rec[a * 3 + 1] +
                                cd.rec[a * 3 + 2] * cd.rec[a * 3 + 2]);
    cd.lrange[a] = (int)std::ceil(rcut * bn / (2.0 * M_PI)) + 1;
  }
  cd.orthorhombic = (A[1] == 0 && A[2] == 0 && A[3] == 0 && A[5] == 0 && A[6] == 0 && A[7] == 0) ? 1 : 0;
  int st = upload_basis(h);
  if (st != ISDF_OK) {
    isdf_destroy(h);
    return st;
  }
  *out = h;
  return ISDF_OK;
}

int isdf_build_points(isdf_handle* h, int n_p, uint64_t seed, double chol_tol, int32_t* ip_index_out) {
  if (!h) return ISDF_ERR_ARG;
  LaunchScope ls(h);
  if (int e = check_device(h)) return e;
  if (n_p < 1 || n_p > h->ng) return fail(h, ISDF_ERR_ARG, "n_p=%d outside [1, N_g=%d]", n_p, h->ng);
  if (!(chol_tol >= 0.0)) return fail(h, ISDF_ERR_ARG, "chol_tol must be >= 0");
  StageTimer stt(h, 0, 0.0);
  if (int e = eval_phi(h)) return e;
  const int ng = h->ng, nkao = h->nk * h->nao;
  double2* phi = (double2*)h->buf("phi");
  ENSURE(d, double, "ip_d", ng);
  ENSURE(Lt, double, "ip_Lt", (size_t)n_p * ng);
  ENSURE(piv, int32_t, "ips", n_p);
  ENSURE(chosen, int32_t, "ip_chosen", ng);
  ENSURE(partial, double, "ip_partial", (size_t)kIpSplit * ng);
  ENSURE(scal, double, "ip_scal", 4);
  ENSURE(status, int32_t, "ip_status", 1);
  CK(cudaMemsetAsync(chosen, 0, sizeof(int32_t) * ng, h->st));
  CK(cudaMemsetAsync(status, 0, sizeof(int32_t), h->st));
  CK(cudaMemsetAsync(piv, 0xff, sizeof(int32_t) * n_p, h->st));
  CK(ip_init(h->st, phi, nkao, ng, d, partial));
  for (int j = 0; j < n_p; ++j)
    CK(ip_step(h->st, phi, nkao, ng, j, d, Lt, piv, chosen, partial, kIpSplit, seed, kTieEps, chol_tol,
               scal, status));
  std::vector<int32_t> hp(n_p);
  int32_t hs = 0;
  CK(cudaMemcpyAsync(hp.data(), piv, sizeof(int32_t) * n_p, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(&hs, status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (hs != 0) {
    int found = 0;
    while (found < n_p && hp[found] >= 0) ++found;
    h->has_points = false;
    return fail(h, ISDF_ERR_NUMERIC, "pivoted Cholesky stopped after %d of %d points (residual below tolerance)",
                found, n_p);
  }
  h->np = n_p;
  h->ips = hp;
  if (ip_index_out) std::memcpy(ip_index_out, hp.data(), sizeof(int32_t) * n_p);
  return finish_points(h);
}

int isdf_set_points(isdf_handle* h, int n_p, const int32_t* ip_index) {
  if (!h) return ISDF_ERR_ARG;
  LaunchScope ls(h);
  if (int e = check_device(h)) return e;
  if (!ip_index || n_p < 1 || n_p > h->ng) return fail(h, ISDF_ERR_ARG, "invalid interpolation points");
  std::vector<char> seen(h->ng, 0);
  for (int i = 0; i < n_p; ++i) {
    if (ip_index[i] < 0 || ip_index[i] >= h->ng || seen[ip_index[i]])
      return fail(h, ISDF_ERR_ARG, "point %d (%d) out of range or repeated", i, ip_index[i]);
    seen[ip_index[i]] = 1;
  }
  if (int e = eval_phi(h)) return e;
  ENSURE(piv, int32_t, "ips", n_p);
  CK(cudaMemcpyAsync(piv, ip_index, sizeof(int32_t) * n_p, cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  h->np = n_p;
  h->ips.assign(ip_index, ip_index + n_p);
  return finish_points(h);
}

int isdf_fit_zeta(isdf_handle* h, double solve_tol, int32_t* rank_out) {
  if (!h) return ISDF_ERR_ARG;
  LaunchScope ls(h);
  if (int e = check_device(h)) return e;
  if (!h->has_points) return fail(h, ISDF_ERR_STATE, "isdf_fit_zeta before the interpolation points");
  if (!(solve_tol >= 0.0) || !(solve_tol < 1.0)) return fail(h, ISDF_ERR_ARG, "solve_tol must be in [0, 1)");
  const int nk = h->nk, np = h->np, nao = h->nao, ng = h->ng;
  const KMesh km{{h->cell.kmesh[0], h->cell.kmesh[1], h->cell.kmesh[2]}};
  double2* X = (double2*)h->buf("X");
  double2* phi = (double2*)h->buf("phi");
  const QHalf qh = fit_q_set(km, h->q_sym);
  // algorithmic work: g^k GEMM (all k) + xi = W eta (triangular) at the computed q
  StageTimer stt(h, 1, 8.0 * nk * (double)np * ng * nao + 4.0 * qh.count * (double)np * np * ng);
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  // Pi^q (Eq. 4): G^k_IJ = sum_mu conj(X^k_I mu) X^k_J mu, then the k-convolution
  ENSURE(Pi, double2, "Pi", (size_t)nk * np * np);
  CK(zgemm(h->st, 'R', 'T', np, np, nao, one, X, nao, (int64_t)np * nao, X, nao, (int64_t)np * nao, zero, Pi,
           np, (int64_t)np * np, nk));
  CK(kdft_cols(h->st, Pi, (int64_t)np * np, km, +1, -1, 1, 1.0 / nk));
  // eta^q (Eq. 5): g^k_I(r) = sum_mu conj(X^k_I mu) Phi^k_mu(r), then the k-convolution.
  // In the mixed and FP64_TC paths g runs on the tensor cores with seven exact
  // slices per operand (~2^-48 relative, FP64-class); the FP64 path keeps FP64
  // arithmetic.
  ENSURE(eta, double2, "eta", (size_t)nk * np * ng);
  if (h->prec != ISDF_FP64 && zgemm_emu_supported(nao)) {
    const size_t per_k = zgemm_emu_work_bytes(np, ng, nao, 1);
    const int nkc = (int)std::max<size_t>(1, std::min<size_t>((size_t)nk, ((size_t)4 << 30) / per_k));
    ENSURE(gw, uint8_t, "grid_work_emu", zgemm_emu_work_bytes(np, ng, nao, nkc));
    ENSURE(tcw, int, "tc_words", 4);
    CK(cudaMemsetAsync(tcw, 0, 4 * sizeof(int), h->st));
    for (int k0 = 0; k0 < nk; k0 += nkc) {
      const int nb = std::min(nkc, nk - k0);
      CK(zgemm_emu(h->st, 'R', np, ng, nao, X + (int64_t)k0 * np * nao, nao, (int64_t)np * nao,
                   phi + (int64_t)k0 * nao * ng, ng, (int64_t)nao * ng, eta + (int64_t)k0 * np * ng, ng,
                   (int64_t)np * ng, nb, gw, tcw + 1));
    }
    int tc_err = 0;
    CK(cudaMemcpyAsync(&tc_err, tcw + 1, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (tc_err != 0) return fail(h, ISDF_ERR_TIMEOUT, "tensor-core GEMM of the fit: bounded wait expired (%d)", tc_err);
  } else {
    CK(zgemm(h->st, 'R', 'N', np, ng, nao, one, X, nao, (int64_t)np * nao, phi, ng, (int64_t)nao * ng, zero, eta,
             ng, (int64_t)np * ng, nk));
  }
  // the k-convolution of Algorithm 1 over the grid columns: FP64 in the FP64 path,
  // float-float (~2^-44 relative, FP32 arithmetic) in the others
  if (h->prec == ISDF_FP64)
    CK(kdft_cols(h->st, eta, (int64_t)np * ng, km, +1, -1, 1, 1.0 / nk));
  else
    CK(kdft_cols_zff(h->st, eta, (int64_t)np * ng, km, +1, -1, 1, 1.0 / nk));
  // Pi^q = L L^H (pivoted), W = L_S^{-1}
  ENSURE(LtPi, double2, "LtPi", (size_t)nk * np * np);
  ENSURE(permPi, int32_t, "permPi", (size_t)nk * np);
  ENSURE(rankPi, int32_t, "rankPi", nk);
  ENSURE(dwork, double, "chol_dwork", (size_t)nk * 2 * np);
  ENSURE(W, double2, "W", (size_t)nk * np * np);
  ENSURE(wwork, double2, "W_work", (size_t)nk * np * np);
  ENSURE(xi, double2, "xi", (size_t)nk * np * ng);
  const int64_t pp = (int64_t)np * np;
  for (const auto& r : qh.runs)
    CK(pchol_batched(h->st, Pi + r.first * pp, np, r.second, solve_tol, LtPi + r.first * pp,
                     permPi + (int64_t)r.first * np, rankPi + r.first, dwork + (int64_t)r.first * 2 * np));
  if (!qh.mirror.empty()) {
    ENSURE(mir, int2, "q_mirror", qh.mirror.size());
    CK(cudaMemcpyAsync(mir, qh.mirror.data(), sizeof(int2) * qh.mirror.size(), cudaMemcpyHostToDevice, h->st));
    // conj(Pi^q) has the diagonals of Pi^q, so the same pivot order and rank
    CK(mirror_copy(h->st, permPi, np, mir, (int)qh.mirror.size()));
    CK(mirror_copy(h->st, rankPi, 1, mir, (int)qh.mirror.size()));
  }
  h->ranks.assign(nk, 0);
  CK(cudaMemcpyAsync(h->ranks.data(), rankPi, sizeof(int32_t) * nk, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (rank_out) std::memcpy(rank_out, h->ranks.data(), sizeof(int32_t) * nk);
  for (int q = 0; q < nk; ++q)
    if (h->ranks[q] < 1) return fail(h, ISDF_ERR_NUMERIC, "Pi^q has rank 0 at q=%d", q);
  // xi^q = W eta^q has nonzero rows only below r_q: keep r_max rows per q
  const int rx = *std::max_element(h->ranks.begin(), h->ranks.end());
  const int64_t pg = (int64_t)np * ng, xg = (int64_t)rx * ng;
  for (const auto& r : qh.runs) {
    const int q0 = r.first, nq = r.second;
    CK(trinv_batched(h->st, LtPi + q0 * pp, permPi + (int64_t)q0 * np, rankPi + q0, np, nq, W + q0 * pp,
                     wwork + q0 * pp));
    // xi^q = W eta^q = L_S^{-1} (eta^q rows in pivot order): triangular, gathered
    CK(ztrmm_gather(h->st, rx, ng, wwork + q0 * pp, np, pp, permPi + (int64_t)q0 * np, np, eta + q0 * pg, ng, pg,
                    xi + q0 * xg, ng, xg, nq));
  }
  if (!qh.mirror.empty()) {
    const int2* mir = (const int2*)h->buf("q_mirror");
    CK(mirror_conj(h->st, W, pp, mir, (int)qh.mirror.size()));
    CK(mirror_conj(h->st, xi, xg, mir, (int)qh.mirror.size()));
  }
  h->xi_rows = rx;
  double tri = 0.0;  // triangular xi = W eta over the computed q: r_q^2 / 2 complex MACs per grid point
  for (const auto& r : qh.runs)
    for (int q = r.first; q < r.first + r.second; ++q) tri += (double)h->ranks[q] * h->ranks[q];
  stt.flops = 8.0 * nk * (double)np * ng * nao + 4.0 * tri * ng;
  h->has_fit = true;
  h->has_xi = true;
  h->has_eta = true;
  h->has_coulomb = false;
  return ISDF_OK;
}

int isdf_coulomb_metric(isdf_handle* h, void* V_out) {
  if (!h) return ISDF_ERR_ARG;
  LaunchScope ls(h);
  if (int e = check_device(h)) return e;
  if (!h->has_fit || !h->has_xi) return fail(h, ISDF_ERR_STATE, "isdf_coulomb_metric before isdf_fit_zeta");
  const int nk = h->nk, np = h->np, ng = h->ng;
  const double2 zero = make_double2(0.0, 0.0);
  double2* xi = (double2*)h->buf("xi");
  double2* W = (double2*)h->buf("W");
  const double2* tw = (const double2*)h->buf("grid_tw");
  const KMesh km{{h->cell.kmesh[0], h->cell.kmesh[1], h->cell.kmesh[2]}};
  const QHalf qh = fit_q_set(km, h->q_sym);
  // xi^q has rx = max_q r_q rows (the rest of the rows of W eta^q vanish), so the
  // grid FFT and the Hermitian GEMM run over rx rows and V_xi is zero beyond them
  const int rx = h->xi_rows;
  StageTimer stt(h, 2, 4.0 * qh.count * (double)rx * rx * ng);  // Hermitian V_xi GEMM
  ENSURE(Vxi, double2, "Vxi", (size_t)nk * np * np);
  ENSURE(gwork, uint8_t, "grid_work", grid_coulomb_work_bytes(nk, h->cell));
  const int64_t pp = (int64_t)np * np, xg = (int64_t)rx * ng;
  CK(cudaMemsetAsync(Vxi, 0, sizeof(double2) * (size_t)nk * pp, h->st));
  // FP64 and FP64_TC: FP64 arithmetic (an error in V_xi reaches E unamplified, as
  // P dV_xi P^H with P = M W^T well scaled, so FP64_TC needs more than four slices here)
  if (h->prec != ISDF_MIXED) {
    for (const auto& r : qh.runs) {
      CK(grid_coulomb_fft(h->st, xi + r.first * xg, rx, r.first, r.second, h->cell, tw, gwork));
      CK(zgemm(h->st, 'R', 'T', rx, rx, ng, make_double2(h->volume, 0.0), xi + r.first * xg, ng, xg,
               xi + r.first * xg, ng, xg, zero, Vxi + r.first * pp, np, pp, r.second));
    }
  } else {
    // mixed: xi rows to float-float in place, the grid FFT in float-float, and
    // V_xi = Omega conj(c')c'^T on the tensor cores with four exact slices (~2^-28 relative;
    // an FP32 FFT and GEMM put ~2e-7 into V_xi, which reaches E and the traces as such)
    ENSURE(tcw, int, "tc_words", 4);
    CK(cudaMemsetAsync(tcw, 0, 4 * sizeof(int), h->st));
    const int qcv = vxi_tc_chunk(rx, ng, (size_t)4 << 30);
    ENSURE(vwork, uint8_t, "grid_work_v", vxi_tc_work_bytes(rx, ng, qcv));
    for (const auto& r : qh.runs) {
      ffcomplex* xf = reinterpret_cast<ffcomplex*>(xi + r.first * xg);
      CK(z2ff(h->st, xi + r.first * xg, xf, r.second * xg));
      CK(grid_coulomb_fft_ff(h->st, xf, rx, r.first, r.second, h->cell, tw, gwork));
      CK(vxi_tc(h->st, xf, xg, rx, ng, r.second, h->volume, Vxi + r.first * pp, np, pp, vwork, qcv, tcw + 1));
    }
    int tc_err = 0;
    CK(cudaMemcpyAsync(&tc_err, tcw + 1, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (tc_err != 0)
      return fail(h, ISDF_ERR_TIMEOUT, "tensor-core Coulomb GEMM: bounded device wait expired (code %d)", tc_err);
  }
  if (!qh.mirror.empty()) {
    ENSURE(mir, int2, "q_mirror", qh.mirror.size());
    CK(cudaMemcpyAsync(mir, qh.mirror.data(), sizeof(int2) * qh.mirror.size(), cudaMemcpyHostToDevice, h->st));
    CK(mirror_conj(h->st, Vxi, pp, mir, (int)qh.mirror.size()));
  }
  h->has_xi = false;  // xi was transformed in place (FP64) / is no longer needed
  return coulomb_tail(h, Vxi, V_out);
}

// Coulomb kernel without forming zeta (Eqs. 7-8): V_eta = Omega c'^* c'^T from
// the grid FFT of eta (Eq. 7), then V_xi = conj(W) V_eta W^T, which is
// W^T V_xi conj(W) = conj(Pi^+) V_eta conj(Pi^+) for the kernel of zeta
// (the least-squares solution of Eq. 8).  Always FP64: rounding in V_eta is
// multiplied by cond(Pi) on the way to W.
int isdf_coulomb_metric_eta(isdf_handle* h, void* V_out) {
  if (!h) return ISDF_ERR_ARG;
  LaunchScope ls(h);
  if (int e = check_device(h)) return e;
  if (!h->has_fit || !h->has_eta)
    return fail(h, ISDF_ERR_STATE, "isdf_coulomb_metric_eta needs eta from isdf_fit_zeta (released after fragments)");
  const int nk = h->nk, np = h->np, ng = h->ng;
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  double2* eta = (double2*)h->buf("eta");
  double2* W = (double2*)h->buf("W");
  double2* work = (double2*)h->buf("xi");  // the copy of eta is transformed in place
  const double2* tw = (const double2*)h->buf("grid_tw");
  const KMesh km{{h->cell.kmesh[0], h->cell.kmesh[1], h->cell.kmesh[2]}};
  const QHalf qh = fit_q_set(km, h->q_sym);
  StageTimer stt(h, 2, 4.0 * qh.count * (double)np * np * ng);
  ENSURE(Vxi, double2, "Vxi", (size_t)nk * np * np);
  ENSURE(Veta, double2, "Veta", (size_t)nk * np * np);
  ENSURE(gwork, uint8_t, "grid_work", grid_coulomb_work_bytes(nk, h->cell));
  h->has_xi = false;
  const int64_t pp = (int64_t)np * np, pg = (int64_t)np * ng;
  for (const auto& r : qh.runs) {
    CK(cudaMemcpyAsync(work + r.first * pg, eta + r.first * pg, sizeof(double2) * (size_t)(r.second * pg),
                       cudaMemcpyDeviceToDevice, h->st));
    CK(grid_coulomb_fft(h->st, work + r.first * pg, np, r.first, r.second, h->cell, tw, gwork));
    CK(zgemm(h->st, 'R', 'T', np, np, ng, make_double2(h->volume, 0.0), work + r.first * pg, ng, pg,
             work + r.first * pg, ng, pg, zero, Veta + r.first * pp, np, pp, r.second));
  }
  if (!qh.mirror.empty()) {
    ENSURE(mir, int2, "q_mirror", qh.mirror.size());
    CK(cudaMemcpyAsync(mir, qh.mirror.data(), sizeof(int2) * qh.mirror.size(), cudaMemcpyHostToDevice, h->st));
    CK(mirror_conj(h->st, Veta, pp, mir, (int)qh.mirror.size()));
  }
  // V_xi = conj(W) (V_eta W^T)
  double2* tmp = (double2*)h->ensure("W_work", sizeof(double2) * (size_t)nk * np * np);
  if (!tmp) return fail(h, ISDF_ERR_OOM, "workspace");
  CK(zgemm(h->st, 'N', 'T', np, np, np, one, Veta, np, (int64_t)np * np, W, np, (int64_t)np * np, zero, tmp, np,
           (int64_t)np * np, nk));
  CK(zgemm(h->st, 'R', 'N', np, np, np, one, W, np, (int64_t)np * np, tmp, np, (int64_t)np * np, zero, Vxi, np,
           (int64_t)np * np, nk));
  return coulomb_tail(h, Vxi, V_out);
}

int isdf_fragment_eri(isdf_handle* h, int n_frag, const int32_t* n_orb, const void* const* C,
                      const void* const* gamma, void* const* eri_out, double* ej_out, double* ek_out) {
  if (!h) return ISDF_ERR_ARG;
  LaunchScope ls(h);
  if (int e = check_device(h)) return e;
  if (!h->has_coulomb) return fail(h, ISDF_ERR_STATE, "isdf_fragment_eri before isdf_coulomb_metric");
  if (n_frag < 0 || (n_frag > 0 && (!n_orb || !C))) return fail(h, ISDF_ERR_ARG, "invalid fragment arrays");
  const int nk = h->nk, np = h->np, nao = h->nao;
  const KMesh km{{h->cell.kmesh[0], h->cell.kmesh[1], h->cell.kmesh[2]}};
  const bool mixed = (h->prec == ISDF_MIXED);
  for (int f = 0; f < n_frag; ++f) {
    const int nf = n_orb[f];
    if (nf < 1 || nf > 4096 || !C[f]) return fail(h, ISDF_ERR_ARG, "fragment %d: bad size or NULL C", f);
    if ((int64_t)nf * nf > 65535LL * 64) return fail(h, ISDF_ERR_ARG, "fragment %d too large", f);
  }
  if (n_frag == 0) return ISDF_OK;
  // The q-points whose B^q enter E, their weights folded into L^q, and their runs.
  std::vector<int> qs;
  std::vector<double> sw;
  q_point_set(km, h->q_sym, qs, sw);
  const int nS = (int)qs.size();
  std::vector<std::pair<int, int>> runs;  // (first q, count) of consecutive q-points
  for (int j = 0; j < nS; ++j) {
    if (!runs.empty() && runs.back().first + runs.back().second == qs[j])
      ++runs.back().second;
    else
      runs.push_back({qs[j], 1});
  }
  std::vector<int> slot(nk, -1);  // position of q in the compact order
  for (int j = 0; j < nS; ++j) slot[qs[j]] = j;
  ENSURE(qmap, int, "frag_qmap", nS);
  ENSURE(swd, double, "frag_sw", nk);
  CK(cudaMemcpyAsync(qmap, qs.data(), sizeof(int) * nS, cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(swd, sw.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, h->st));
  const double2* Lq = (const double2*)h->buf("Lq");
  const int64_t pp = (int64_t)np * np;
  // Structural zeros of L^q = W^T L_xi: nonzero rows perm_q[c] (c < r_q, the
  // pivots of Pi^q), nonzero columns J < n_q (the rank of V_xi^q).  B^q = M^q L^q
  // needs only those; rp and nv bound them over the q of the sum.
  int rp = 1, nv = 1;
  double sum_nv = 0.0, sum_rn = 0.0;
  for (int q : qs) {
    rp = std::max(rp, (int)h->ranks[q]);
    nv = std::max(nv, (int)h->ranks_v[q]);
    sum_nv += h->ranks_v[q];
    sum_rn += (double)h->ranks[q] * h->ranks_v[q];
  }
  const int nj = (int)std::min<int64_t>(np, ((int64_t)nv + 3) / 4 * 4);  // columns of B^q
  const int32_t* permPi = (const int32_t*)h->buf("permPi");
  const int32_t* rankPi = (const int32_t*)h->buf("rankPi");
  // The fragments go one after the other on the stream with no host
  // synchronisation in between: each writes its traces into its slot of a
  // device array, and the bounded-wait error word of the tensor-core kernels is
  // read once at the end.
  const bool any_tr = (ej_out || ek_out) && gamma;
  ENSURE(trall, double, "frag_traces", 4 * (size_t)n_frag);
  ENSURE(tcw, int, "tc_words", 4);
  CK(cudaMemsetAsync(trall, 0, sizeof(double) * 4 * (size_t)n_frag, h->st));
  CK(cudaMemsetAsync(tcw, 0, 4 * sizeof(int), h->st));
  // FP64_TC: the grouped tensor-core path in float-float with more exact slices,
  // where B = M L fits its exact accumulation (2 r_q <= 576); else FP64 arithmetic
  const bool tc64 = (h->prec == ISDF_FP64_TC) && mlgemm5_tc_supported(rp);
  if (!mixed && !tc64) {
    for (int f = 0; f < n_frag; ++f) {
      const int nf = n_orb[f];
      const int64_t n2 = (int64_t)nf * nf;
      const int64_t sq = n2 * np;  // q stride of M
      const double2* Cf = (const double2*)C[f];
      double* trf = trall + 4 * (int64_t)f;
      double2* trpart = nullptr;
      const bool want_tr = any_tr && gamma[f];
      if (want_tr) {
        trpart = (double2*)h->ensure("frag_traces_part", sizeof(double2) * 2 * (size_t)n2);
        if (!trpart) return fail(h, ISDF_ERR_OOM, "traces workspace");
      }
      const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
      double2* X = (double2*)h->buf("X");
      ENSURE(Lw, double2, "frag_Lw", (size_t)nk * pp);
      ENSURE(T, double2, "frag_T", (size_t)nk * np * nf);
      ENSURE(M, double2, "frag_M", (size_t)nk * sq);
      ENSURE(B, double2, "frag_B", (size_t)n2 * nS * nj);
      ENSURE(E, double2, "frag_E", (size_t)n2 * n2);
      if (f == 0) CK(scale_blocks(h->st, Lq, pp, nk, swd, Lw));
      {
        StageTimer stt(h, 3, frag_m_flops(nk, np, nf, nao, km));
        CK(zgemm(h->st, 'N', 'N', np, nf, nao, one, X, nao, (int64_t)np * nao, Cf, nf, (int64_t)nao * nf, zero, T,
                 nf, (int64_t)np * nf, nk));
        CK(kdft_cols(h->st, T, (int64_t)np * nf, km, +1, +1, 0, 1.0));
        CK(pair_products(h->st, T, nk, np, nf, M));
        CK(kdft_cols(h->st, M, n2 * np, km, +1, +1, 0, 1.0 / nk));
      }
      {
        // B = [w_q^{1/2} M^q L^q]_{q in S}, compact: B[a][slot(q) nj + J], the nj
        // nonzero columns of L^q
        StageTimer stt(h, 4, 8.0 * (double)n2 * np * sum_nv);
        for (const auto& r : runs)
          CK(zgemm(h->st, 'N', 'N', (int)n2, nj, np, one, M + r.first * sq, np, sq, Lw + r.first * pp, np, pp, zero,
                   B + (int64_t)slot[r.first] * nj, (int64_t)nS * nj, nj, r.second));
      }
      {
        StageTimer stt(h, 5, 4.0 * (double)n2 * n2 * sum_nv);
        CK(zgemm(h->st, 'N', 'C', (int)n2, (int)n2, nS * nj, one, B, (int64_t)nS * nj, 0, B, (int64_t)nS * nj, 0,
                 zero, E, n2, 0, 1));
        if (h->q_sym) CK(eri_swapconj_sym(h->st, E, nf));
      }
      if (eri_out && eri_out[f]) CK(eri_permute(h->st, E, nf, 1.0 / nk, (double2*)eri_out[f]));
      if (want_tr) CK(eri_traces(h->st, E, nf, 1.0 / nk, (const double2*)gamma[f], trf, trpart));
    }
  } else {
    const float2 one = make_float2(1.f, 0.f), zero = make_float2(0.f, 0.f);
    float2* Xf = tc64 ? nullptr : (float2*)h->buf("X_f");
    const double2* Xz = (const double2*)h->buf("X");
    // element bytes of the pair rows Z (float / float-float) and of M^q, B^q
    const size_t zsz = tc64 ? sizeof(ffloat) : sizeof(float), msz = tc64 ? sizeof(ffcomplex) : sizeof(float2);
    // B = M L on the tensor cores (three remainder slices; five exact ones in FP64_TC) when the
    // 2 r_q gathered columns fit their exact accumulation, else on the
    // compensated SIMT GEMM
    const bool tc_ml = tc64 || mlgemm_tc_supported(rp);
    float2* Lwf = nullptr;
    void* lsl = nullptr;
    int* lexp = nullptr;
    if (tc_ml) {
      lsl = h->ensure_evict("frag_Lsl", tc64 ? mlgemm5_tc_lslice_bytes(nk, rp, nj) : mlgemm_tc_lslice_bytes(nk, rp, nj));
      lexp = (int*)h->ensure_evict("frag_Lexp",
                                   sizeof(int) * (size_t)nk * (tc64 ? mlgemm5_tc_nj_pad(nj) : mlgemm_tc_nj_pad(nj)));
      if (!lsl || !lexp) return fail(h, ISDF_ERR_OOM, "device allocation of the slices of L failed");
      if (tc64)
        CK(mlgemm5_tc_prepare(h->st, Lq, swd, nk, np, permPi, rankPi, rp, nj, lsl, lexp));
      else
        CK(mlgemm_tc_prepare(h->st, Lq, swd, nk, np, permPi, rankPi, rp, nj, lsl, lexp));
    } else {
      Lwf = (float2*)h->ensure_evict("frag_Lwf", sizeof(float2) * (size_t)nk * pp);
      if (!Lwf) return fail(h, ISDF_ERR_OOM, "device allocation of frag_Lwf failed");
      CK(scale_blocks_f(h->st, Lq, pp, nk, swd, Lwf));
    }
    ENSURE(qslot_d, int, "frag_qslot", nk);
    CK(cudaMemcpyAsync(qslot_d, slot.data(), nk * sizeof(int), cudaMemcpyHostToDevice, h->st));
    const int64_t ldB = tc_ml ? nj : np;
    // Groups of fragments contracted together: fragments whose lower triangle of
    // 128 x 128 tiles fills few waves of the GPU go with others of their kind,
    // their rows stacked (each block padded to a tile boundary) so that one launch
    // of each kernel covers the group and the tiles of all its diagonal blocks;
    // a group never needs more scratch than the largest fragment alone.
    const std::vector<std::vector<int>> groups = fragment_groups(n_frag, n_orb, nk, nS, np, tc64 ? 2.0 : 1.0);
    for (const auto& grp : groups) {
      // rows of each fragment inside the stacked block; padding rows are zero
      std::vector<int64_t> row0(grp.size());
      int64_t rows = 0;
      for (size_t i = 0; i < grp.size(); ++i) {
        const int64_t n2f = (int64_t)n_orb[grp[i]] * n_orb[grp[i]];
        row0[i] = rows;
        rows += (i + 1 < grp.size()) ? (n2f + 127) / 128 * 128 : n2f;
      }
      const int64_t sq = rows * np;  // q stride of M
      int nfmax = 0;
      double flops3 = 0.0, flops4 = 0.0, flops5 = 0.0;
      for (int f : grp) {
        const int64_t n2f = (int64_t)n_orb[f] * n_orb[f];
        nfmax = std::max(nfmax, (int)n_orb[f]);
        flops3 += frag_m_flops(nk, np, n_orb[f], nao, km);
        flops4 += 8.0 * (double)n2f * (tc_ml ? sum_rn : (double)np * sum_nv);
        flops5 += 2.0 * (double)n2f * (double)(n2f + 1) * sum_nv;
      }
      const int64_t n2max = (int64_t)nfmax * nfmax;
      // T^k = X^k C^k: complex64 (mixed) or complex128 then float-float in place (FP64_TC)
      ENSURE(Cff, float2, "frag_Cf", tc64 ? 1 : (size_t)nk * nao * nfmax);
      ENSURE(T, float2, "frag_T", (size_t)nk * np * nfmax * (tc64 ? 2 : 1));
      // real pair rows Z(R) of the time-reversal basis, and M^q (then B^q) of the
      // q of the sum, stored by their position in it
      ENSURE(Zr, uint8_t, "frag_Zr", zsz * (size_t)nk * sq);
      ENSURE(M, uint8_t, "frag_Mf", msz * (size_t)nS * sq);
      float* Zr_f = reinterpret_cast<float*>(Zr);
      ffloat* Zr_ff = reinterpret_cast<ffloat*>(Zr);
      float2* M_f = reinterpret_cast<float2*>(M);
      ffcomplex* M_ff = reinterpret_cast<ffcomplex*>(M);
      ENSURE(trpart, double2, "frag_traces_part", std::max<size_t>(2 * (size_t)n2max, syrk_tc_eri_part_count()));
      // tiles of every fragment's diagonal block, in the autotuned band order
      std::vector<int2>& tl = h->tiles_host;
      std::vector<int>& tof = h->tile_of_host;
      std::vector<int64_t> tof_off(grp.size());
      auto build_tiles = [&](int band) {
        tl.clear();
        tof.clear();
        for (size_t i = 0; i < grp.size(); ++i) {
          const int64_t n2f = (int64_t)n_orb[grp[i]] * n_orb[grp[i]];
          std::vector<int2> t;
          std::vector<int> of;
          syrk_tc_tiles(n2f, t, of, band);
          const int t0 = (int)(row0[i] / 128), base = (int)tl.size();
          for (const int2& x : t) tl.push_back(make_int2(x.x + t0, x.y + t0));
          tof_off[i] = (int64_t)tof.size();
          for (int v : of) tof.push_back(v < 0 ? -1 : v + base);
        }
      };
      build_tiles(12);
      std::vector<int2>& orb = h->orb_host;
      std::vector<int64_t> orb_off(grp.size());
      orb.clear();
      for (size_t i = 0; i < grp.size(); ++i) {
        std::vector<int2> o;
        pair_orbits(n_orb[grp[i]], o);
        orb_off[i] = (int64_t)orb.size();
        orb.insert(orb.end(), o.begin(), o.end());
      }
      // B^q = w_q^{1/2} M^q L^q overwrites M^q (row pitch nj on the tensor-core
      // path, np through Bc on the SIMT path), qc q-points at a time; E' then
      // takes the rows of B^q in chunks of qc positions (fp16 slices of 2 qc nj
      // columns).  qc fits both slice buffers in the workspace limit.
      auto syrk_split_bytes = [&](int64_t kc) {
        return tc64 ? syrk4_tc_split_bytes(rows, kc) : syrk_tc_split_bytes(rows, kc);
      };
      auto ml_split_bytes = [&](int nq) -> size_t {
        if (!tc_ml) return 0;
        return tc64 ? mlgemm5_tc_split_bytes(rows, rp, nq) : mlgemm_tc_split_bytes(rows, rp, nq);
      };
      const size_t per_q = std::max(syrk_split_bytes(nj), ml_split_bytes(1));
      const int qc = (int)std::max<int64_t>(1, std::min<int64_t>(nS, (int64_t)(h->split_budget / per_q)));
      ENSURE(split, uint8_t, "tc_split", std::max(syrk_split_bytes((int64_t)qc * nj), ml_split_bytes(qc)));
      float2* Bc = nullptr;
      if (!tc_ml) {
        Bc = (float2*)h->ensure_evict("frag_Bc", sizeof(float2) * (size_t)qc * sq);
        if (!Bc) return fail(h, ISDF_ERR_OOM, "device allocation of frag_Bc failed");
      }
      ENSURE(rexp, int, "tc_rowexp", rows);
      ENSURE(tiles_d, int2, "tc_tiles", tl.size());
      ENSURE(tile_of_d, int, "tc_tile_of", tof.size());
      ENSURE(orb_d, int2, "tc_orbits", orb.size());
      ENSURE(ws, uint8_t, "tc_ws", syrk_tc_ws_bytes((int64_t)tl.size()));
      CK(cudaMemcpyAsync(tiles_d, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice, h->st));
      CK(cudaMemcpyAsync(tile_of_d, tof.data(), tof.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
      CK(cudaMemcpyAsync(orb_d, orb.data(), orb.size() * sizeof(int2), cudaMemcpyHostToDevice, h->st));
      {
        StageTimer stt(h, 3, flops3);
        for (size_t i = 0; i < grp.size(); ++i) {
          const int f = grp[i], nf = n_orb[f];
          const int64_t n2f = (int64_t)nf * nf;
          if (tc64) {
            // T = X C FP64-class (tensor cores, seven exact slices; FP64 beyond N_AO = 64),
            // then float-float in place for the DFT and the pair rows
            double2* Tz = reinterpret_cast<double2*>(T);
            if (zgemm_emu_supported(nao)) {
              ENSURE(tew, uint8_t, "frag_T_emu", zgemm_emu_work_bytes(np, nfmax, nao, nk));
              CK(zgemm_emu(h->st, 'N', np, nf, nao, Xz, nao, (int64_t)np * nao, (const double2*)C[f], nf,
                           (int64_t)nao * nf, Tz, nf, (int64_t)np * nf, nk, tew, tcw + 1));
            } else {
              CK(zgemm(h->st, 'N', 'N', np, nf, nao, make_double2(1.0, 0.0), Xz, nao, (int64_t)np * nao,
                       (const double2*)C[f], nf, (int64_t)nao * nf, make_double2(0.0, 0.0), Tz, nf,
                       (int64_t)np * nf, nk));
            }
            ffcomplex* Tff = reinterpret_cast<ffcomplex*>(Tz);
            CK(z2ff(h->st, Tz, Tff, (int64_t)nk * np * nf));
            CK(kdft_cols_ff(h->st, Tff, (int64_t)np * nf, km, +1, +1, 0, 1.0));
            CK(pair_products_real_ff(h->st, Tff, nk, np, nf, Zr_ff, row0[i], rows));
          } else {
            CK(z2c(h->st, (const double2*)C[f], Cff, (int64_t)nk * nao * nf));
            CK(cgemm(h->st, 'N', 'N', np, nf, nao, one, Xf, nao, (int64_t)np * nao, Cff, nf, (int64_t)nao * nf,
                     zero, T, nf, (int64_t)np * nf, nk));
            CK(kdft_cols_f(h->st, T, (int64_t)np * nf, km, +1, +1, 0, 1.f));
            // pair rows in the time-reversal basis are real: Z(R) in FP32
            CK(pair_products_real_f(h->st, T, nk, np, nf, Zr_f, row0[i], rows));
          }
          const int64_t pad = (i + 1 < grp.size()) ? row0[i + 1] - row0[i] - n2f : 0;
          if (pad > 0)
            CK(cudaMemset2DAsync(Zr + zsz * (size_t)((row0[i] + n2f) * np), zsz * (size_t)sq, 0,
                                 zsz * (size_t)(pad * np), nk, h->st));
        }
        // the R -> q DFT keeps only the q of the sum (M^{-q} = conj(M^q))
        if (tc64)
          CK(kdft_real_ff(h->st, Zr_ff, M_ff, sq, km, +1, 1.0 / nk, qslot_d));
        else
          CK(kdft_real_f(h->st, Zr_f, M_f, sq, km, +1, 1.f / nk, qslot_d));
      }
      {
        StageTimer stt(h, 4, flops4);
        if (tc64) {
          // as below, five exact slices of the float-float M and of L, B in float-float
          CK(mlgemm5_tc_rowscale(h->st, M_ff, sq, np, qmap, nS, permPi, rankPi, rp, rows, rexp));
          for (int j0 = 0; j0 < nS; j0 += qc)
            CK(mlgemm5_tc_chunk(h->st, M_ff, sq, qmap, rows, np, permPi, rankPi, rp, nj, j0, std::min(qc, nS - j0),
                                rexp, split, lsl, lexp, nk, tcw + 1));
        } else if (tc_ml) {
          // row exponents of the gathered M over the q of the sum, then B^q = M^q L^q
          // over M^q, q-chunk by q-chunk
          CK(mlgemm_tc_rowscale(h->st, M_f, sq, np, qmap, nS, permPi, rankPi, rp, rows, rexp));
          for (int j0 = 0; j0 < nS; j0 += qc)
            CK(mlgemm_tc_chunk(h->st, M_f, sq, qmap, rows, np, permPi, rankPi, rp, nj, j0, std::min(qc, nS - j0),
                               rexp, split, lsl, lexp, nk, tcw + 1));
        } else {
          // consecutive q of a run sit at consecutive positions
          for (const auto& r : runs)
            for (int q0 = r.first; q0 < r.first + r.second; q0 += qc) {
              const int nq = std::min(qc, r.first + r.second - q0);
              const int64_t j = slot[q0];
              CK(cgemm(h->st, 'N', 'N', (int)rows, np, np, one, M_f + j * sq, np, sq, Lwf + q0 * pp, np, pp, zero,
                       Bc, np, sq, nq));
              CK(cudaMemcpyAsync(M_f + j * sq, Bc, sizeof(float2) * (size_t)nq * sq, cudaMemcpyDeviceToDevice,
                                 h->st));
            }
        }
      }
      {
        // E' = c sum_{q in S} [Re R^q, Im R^q][Re R^q, Im R^q]^T over the rows of B^q in the
        // time-reversal basis (real symmetric, lower-triangle tiles of each diagonal block),
        // then E = W E' W^H per fragment; c = 2 with the pairing, 1 over every q
        StageTimer stt(h, 5, flops5);
        if (tc64)
          CK(syrk4_tc_rowscale(h->st, M_ff, sq, ldB, nj, nS, rows, rexp));
        else
          CK(syrk_tc_rowscale(h->st, M_f, sq, ldB, nj, nullptr, nS, rows, rexp));
        // per-row sums of the left-out diagonal products, accumulated chunk by chunk
        ENSURE(dcorr, double, "tc_diag_corr", rows);
        CK(cudaMemsetAsync(dcorr, 0, sizeof(double) * (size_t)rows, h->st));
        const int nq0 = std::min(qc, nS);
        // FP64_TC has one pipeline (no tuning); the band order of the mixed default
        const TileSchedule sch = tc64 ? TileSchedule{0, 12} : tuned_schedule(h, (int64_t)tl.size(), [&](int cfg, int b) -> int {
          build_tiles(b);
          if (cudaMemcpyAsync(tiles_d, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice, h->st) !=
              cudaSuccess)
            return -1;
          return syrk_tc_chunk(h->st, M_f, sq, ldB, nj, nullptr, rows, 0, nq0, rexp, split, tiles_d,
                               (int)tl.size(), ws, 0, tcw + 1, cfg) == cudaSuccess ? 0 : -1;
        });
        if (sch.band < 0) return fail(h, ISDF_ERR_CUDA, "tile-schedule tuning launch failed");
        build_tiles(sch.band);
        CK(cudaMemcpyAsync(tiles_d, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice, h->st));
        CK(cudaMemcpyAsync(tile_of_d, tof.data(), tof.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
        for (int j0 = 0; j0 < nS; j0 += qc) {
          const int nq = std::min(qc, nS - j0);
          double nv_chunk = 0.0;  // the chunk's share of the algorithmic flops
          for (int j = j0; j < j0 + nq; ++j) nv_chunk += h->ranks_v[qs[j]];
          if (tc64) {
            CK(syrk4_tc_split(h->st, M_ff, sq, ldB, nj, rows, j0, nq, rexp, split, dcorr));
            StageTimer stk(h, 6, flops5 * nv_chunk / std::max(sum_nv, 1.0));
            CK(syrk4_tc_mma(h->st, split, rows, nq, nj, tiles_d, (int)tl.size(), ws, j0 > 0, tcw + 1));
          } else {
            CK(syrk_tc_split(h->st, M_f, sq, ldB, nj, nullptr, rows, j0, nq, rexp, split, dcorr));
            StageTimer stk(h, 6, flops5 * nv_chunk / std::max(sum_nv, 1.0));
            CK(syrk_tc_mma(h->st, split, rows, nq, nj, tiles_d, (int)tl.size(), ws, j0 > 0, tcw + 1, sch.cfg));
          }
        }
        // E = W E' W^H per fragment, written straight to the caller's ERIs (chemist's
        // order) with the FP64 traces accumulated on the way
        for (size_t i = 0; i < grp.size(); ++i) {
          const int f = grp[i];
          const double sc = (h->q_sym ? 2.0 : 1.0) / nk;
          const double2* gf = any_tr ? (const double2*)gamma[f] : nullptr;
          if (tc64)
            CK(syrk_tc_finish_eri_z(h->st, ws, (int)tl.size(), tile_of_d + tof_off[i], orb_d + orb_off[i],
                                    n_orb[f], rexp + row0[i], dcorr + row0[i], sc,
                                    eri_out ? (double2*)eri_out[f] : nullptr, gf, trpart, trall + 4 * (int64_t)f));
          else
            CK(syrk_tc_finish_eri(h->st, ws, (int)tl.size(), tile_of_d + tof_off[i], orb_d + orb_off[i], n_orb[f],
                                  rexp + row0[i], dcorr + row0[i], sc, eri_out ? (float2*)eri_out[f] : nullptr, gf,
                                  trpart, trall + 4 * (int64_t)f));
        }
      }
    }
  }
  std::vector<double> hv(4 * (size_t)n_frag, 0.0);
  int tc_err = 0;
  if (any_tr) CK(cudaMemcpyAsync(hv.data(), trall, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(&tc_err, tcw + 1, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (tc_err != 0)
    return fail(h, ISDF_ERR_TIMEOUT, "tensor-core contraction: bounded device wait expired (code %d)", tc_err);
  for (int f = 0; f < n_frag; ++f) {
    if (ej_out) ej_out[f] = hv[4 * (size_t)f];
    if (ek_out) ek_out[f] = hv[4 * (size_t)f + 1];
  }
  return ISDF_OK;
}

int isdf_ao_eri(isdf_handle* h, int n_quartet, const int32_t* quartets, void* out) {
  if (!h) return ISDF_ERR_ARG;
  LaunchScope ls(h);
  if (int e = check_device(h)) return e;
  if (!h->has_coulomb) return fail(h, ISDF_ERR_STATE, "isdf_ao_eri before the Coulomb metric");
  if (n_quartet < 0 || (n_quartet > 0 && (!quartets || !out))) return fail(h, ISDF_ERR_ARG, "invalid quartet arrays");
  const int nk = h->nk, np = h->np, nao = h->nao;
  const int* km = h->cell.kmesh;
  auto coords = [&](int k, int m[3]) {
    m[0] = k / (km[1] * km[2]);
    m[1] = (k / km[2]) % km[1];
    m[2] = k % km[2];
  };
  auto flat = [&](const int m[3]) {
    return ((((m[0] % km[0]) + km[0]) % km[0]) * km[1] + (((m[1] % km[1]) + km[1]) % km[1])) * km[2] +
           (((m[2] % km[2]) + km[2]) % km[2]);
  };
  std::vector<int> qv(n_quartet);
  for (int n = 0; n < n_quartet; ++n) {
    const int32_t* k = quartets + 4 * n;
    for (int i = 0; i < 4; ++i)
      if (k[i] < 0 || k[i] >= nk) return fail(h, ISDF_ERR_ARG, "quartet %d: k index out of range", n);
    int m1[3], m2[3], m3[3], m4[3], d[3], s4[3];
    coords(k[0], m1), coords(k[1], m2), coords(k[2], m3), coords(k[3], m4);
    for (int a = 0; a < 3; ++a) {
      d[a] = m1[a] - m2[a];
      s4[a] = m3[a] + d[a];
    }
    if (flat(s4) != k[3])
      return fail(h, ISDF_ERR_ARG, "quartet %d does not conserve crystal momentum (k1 - k2 != k4 - k3)", n);
    qv[n] = flat(d);
  }
  const int64_t nao2 = (int64_t)nao * nao, pp = (int64_t)np * np, pa = (int64_t)np * nao;
  double2* X = (double2*)h->buf("X");
  double2* Lq = (double2*)h->buf("Lq");
  ENSURE(A, double2, "ao_pairs_a", (size_t)np * nao2);
  ENSURE(Cc, double2, "ao_pairs_c", (size_t)np * nao2);
  ENSURE(U, double2, "ao_u", (size_t)np * nao2);
  ENSURE(Wm, double2, "ao_w", (size_t)np * nao2);
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  for (int n = 0; n < n_quartet; ++n) {
    const int32_t* k = quartets + 4 * n;
    const double2* L = Lq + qv[n] * pp;
    CK(ao_pairs(h->st, X + k[0] * pa, X + k[1] * pa, np, nao, A));
    CK(ao_pairs(h->st, X + k[2] * pa, X + k[3] * pa, np, nao, Cc));
    // (mu nu|lam sig) = Nk A^T V^Q C with V^Q = L L^H: (L^T A)^T (L^H C)
    CK(zgemm(h->st, 'T', 'N', np, (int)nao2, np, one, L, np, 0, A, nao2, 0, zero, U, nao2, 0, 1));
    CK(zgemm(h->st, 'C', 'N', np, (int)nao2, np, one, L, np, 0, Cc, nao2, 0, zero, Wm, nao2, 0, 1));
    CK(zgemm(h->st, 'T', 'N', (int)nao2, (int)nao2, np, make_double2((double)nk, 0.0), U, nao2, 0, Wm, nao2, 0,
             zero, (double2*)out + (int64_t)n * nao2 * nao2, nao2, 0, 1));
  }
  CK(cudaStreamSynchronize(h->st));
  return ISDF_OK;
}

int isdf_sos_polarizability(isdf_handle* h, const void* C, int n_mo, int n_occ, const double* eps, double tau,
                            void* chi_out, double* s_out) {
  if (!h) return ISDF_ERR_ARG;
  LaunchScope ls(h);
  if (int e = check_device(h)) return e;
  if (!h->has_coulomb) return fail(h, ISDF_ERR_STATE, "isdf_sos_polarizability before the Coulomb metric");
  if (!C || !eps || n_mo < 1 || n_occ < 1 || n_occ >= n_mo || !(tau >= 0.0) || !std::isfinite(tau))
    return fail(h, ISDF_ERR_ARG, "isdf_sos_polarizability: need C, eps, 0 < n_occ < n_mo and finite tau >= 0");
  const int nk = h->nk, np = h->np, nao = h->nao, nvir = n_mo - n_occ;
  const int64_t pp = (int64_t)np * np;
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  double2* X = (double2*)h->buf("X");
  double2* Lq = (double2*)h->buf("Lq");
  ENSURE(epsd, double, "sos_eps", (size_t)nk * n_mo);
  ENSURE(Y, double2, "sos_y", (size_t)nk * np * n_mo);
  ENSURE(Yo, double2, "sos_yo", (size_t)nk * np * n_occ);
  ENSURE(Yv, double2, "sos_yv", (size_t)nk * np * nvir);
  ENSURE(Go, double2, "sos_go", (size_t)nk * pp);
  ENSURE(Gv, double2, "sos_gv", (size_t)nk * pp);
  ENSURE(chi_w, double2, "sos_chi", (size_t)nk * pp);
  ENSURE(Vq, double2, "sos_v", (size_t)nk * pp);
  ENSURE(T1, double2, "sos_t1", (size_t)nk * pp);
  ENSURE(part, double, "sos_part", nk);
  double2* chi = chi_out ? (double2*)chi_out : chi_w;
  CK(cudaMemcpyAsync(epsd, eps, sizeof(double) * (size_t)nk * n_mo, cudaMemcpyHostToDevice, h->st));
  // Y^k = X^k C^k (orbital values at the points, Eq. 14)
  CK(zgemm(h->st, 'N', 'N', np, n_mo, nao, one, X, nao, (int64_t)np * nao, (const double2*)C, n_mo,
           (int64_t)nao * n_mo, zero, Y, n_mo, (int64_t)np * n_mo, nk));
  // Go^k = Y_occ e^{+tau eps_i} Y_occ^H,  Gv^k = Y_vir e^{-tau eps_a} Y_vir^H (Eq. 15)
  CK(scale_cols(h->st, Y, nk, np, n_mo, 0, n_occ, epsd, +tau, Yo));
  CK(scale_cols(h->st, Y, nk, np, n_mo, n_occ, nvir, epsd, -tau, Yv));
  CK(zgemm(h->st, 'N', 'C', np, np, n_occ, one, Yo, n_occ, (int64_t)np * n_occ, Y, n_mo, (int64_t)np * n_mo, zero,
           Go, np, pp, nk));
  CK(zgemm(h->st, 'N', 'C', np, np, nvir, one, Yv, nvir, (int64_t)np * nvir, Y + n_occ, n_mo, (int64_t)np * n_mo,
           zero, Gv, np, pp, nk));
  // chi^Q_{IK} = sum_k Go^k_{KI} Gv^{k-Q}_{IK} (Eq. 13) by the convolution theorem, as
  // Algorithm 1 does for Pi^q: with hat(a)(R) = sum_k a(k) e^{+ik.R} and
  // check(b)(R) = sum_k b(k) e^{-ik.R},  chi = (1/Nk) DFT_-( hat(Go)^T o check(Gv) )
  const KMesh km{{h->cell.kmesh[0], h->cell.kmesh[1], h->cell.kmesh[2]}};
  CK(kdft_cols(h->st, Go, pp, km, +1, +1, 0, 1.0));
  CK(kdft_cols(h->st, Gv, pp, km, -1, -1, 0, 1.0));
  CK(hadamard_t(h->st, Go, Gv, np, nk, chi));
  CK(kdft_cols(h->st, chi, pp, km, -1, -1, 0, 1.0 / nk));
  if (s_out) {
    // S = Nk^2 sum_Q tr[conj(V^Q) chi^Q conj(V^Q) (chi^{-Q})^T], V^Q = L^Q L^Q^H (Eq. 12)
    CK(zgemm(h->st, 'N', 'C', np, np, np, one, Lq, np, pp, Lq, np, pp, zero, Vq, np, pp, nk));
    CK(zgemm(h->st, 'R', 'N', np, np, np, one, Vq, np, pp, chi, np, pp, zero, T1, np, pp, nk));
    CK(zgemm(h->st, 'N', 'R', np, np, np, one, T1, np, pp, Vq, np, pp, zero, Go, np, pp, nk));  // Go reused
    CK(sos_trace_parts(h->st, Go, chi, h->cell.kmesh, np, part));
    std::vector<double> hp(nk);
    CK(cudaMemcpyAsync(hp.data(), part, sizeof(double) * nk, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    double S = 0.0;
    for (int q = 0; q < nk; ++q) S += hp[q];
    *s_out = (double)nk * (double)nk * S;
  }
  CK(cudaStreamSynchronize(h->st));
  return ISDF_OK;
}

int isdf_exchange(isdf_handle* h, const void* P, void* K_out) {
  if (!h || !P || !K_out) return fail(h, ISDF_ERR_ARG, "isdf_exchange: NULL argument");
  LaunchScope ls(h);
  if (int e = check_device(h)) return e;
  if (!h->has_coulomb) return fail(h, ISDF_ERR_STATE, "isdf_exchange before the Coulomb metric");
  const int nk = h->nk, np = h->np, nao = h->nao;
  const KMesh km{{h->cell.kmesh[0], h->cell.kmesh[1], h->cell.kmesh[2]}};
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  double2* X = (double2*)h->buf("X");
  double2* Lq = (double2*)h->buf("Lq");
  ENSURE(rho, double2, "kx_rho", (size_t)nk * np * np);
  ENSURE(Vd, double2, "kx_V", (size_t)nk * np * np);
  ENSURE(t1, double2, "kx_t1", (size_t)nk * np * (nao > np ? nao : np));
  // rho^k = X^k P^k X^k^H
  CK(zgemm(h->st, 'N', 'N', np, nao, nao, one, X, nao, (int64_t)np * nao, (const double2*)P, nao,
           (int64_t)nao * nao, zero, t1, nao, (int64_t)np * nao, nk));
  CK(zgemm(h->st, 'N', 'C', np, np, nao, one, t1, nao, (int64_t)np * nao, X, nao, (int64_t)np * nao, zero, rho, np,
           (int64_t)np * np, nk));
  // V^q = L^q L^q^H
  CK(zgemm(h->st, 'N', 'C', np, np, np, one, Lq, np, (int64_t)np * np, Lq, np, (int64_t)np * np, zero, Vd, np,
           (int64_t)np * np, nk));
  // Gamma^k = sum_k' (V^{k'-k})^T o rho^{k'}: DFT_- V, DFT_+ rho, transposed product, DFT_- / Nk
  CK(kdft_cols(h->st, Vd, (int64_t)np * np, km, -1, -1, 0, 1.0));
  CK(kdft_cols(h->st, rho, (int64_t)np * np, km, +1, +1, 0, 1.0));
  CK(hadamard_t(h->st, Vd, rho, np, nk, rho));
  CK(kdft_cols(h->st, rho, (int64_t)np * np, km, -1, -1, 0, 1.0 / nk));
  // K^k = -(1/Nk) X^k^H Gamma^k X^k
  CK(zgemm(h->st, 'N', 'N', np, nao, np, one, rho, np, (int64_t)np * np, X, nao, (int64_t)np * nao, zero, t1, nao,
           (int64_t)np * nao, nk));
  CK(zgemm(h->st, 'C', 'N', nao, nao, np, make_double2(-1.0 / nk, 0.0), X, nao, (int64_t)np * nao, t1, nao,
           (int64_t)np * nao, zero, (double2*)K_out, nao, (int64_t)nao * nao, nk));
  CK(cudaStreamSynchronize(h->st));
  return ISDF_OK;
}

int isdf_set_time_reversal(isdf_handle* h, int enable) {
  if (!h) return ISDF_ERR_ARG;
  h->q_sym = (enable != 0);
  return ISDF_OK;
}

int isdf_set_autotune(isdf_handle* h, int enable) {
  if (!h) return ISDF_ERR_ARG;
  h->autotune = (enable != 0);
  return ISDF_OK;
}

int isdf_set_tile_schedule(isdf_handle* h, int pipeline, int band) {
  if (!h) return ISDF_ERR_ARG;
  if ((pipeline != 0 && pipeline != 1) || band < 1 || band > 64)
    return fail(h, ISDF_ERR_ARG, "tile schedule: pipeline must be 0 or 1 and band in [1, 64]");
  h->autotune = false;
  h->fixed_cfg = pipeline;
  h->fixed_band = band;
  return ISDF_OK;
}

int isdf_autotune_report(const isdf_handle* h, char* buf, size_t len) {
  if (!h || !buf || len == 0) return ISDF_ERR_ARG;
  std::string r = "[";
  for (size_t i = 0; i < h->tune_log.size(); ++i) {
    const auto& e = h->tune_log[i];
    char b[200];
    snprintf(b, sizeof(b), "%s{\"tiles\": %lld, \"pipeline\": %d, \"band\": %d, \"ms\": [%.3f, %.3f, %.3f, %.3f]}",
             i ? ", " : "", (long long)e.ntiles, e.cfg, e.band, e.ms[0], e.ms[1], e.ms[2], e.ms[3]);
    r += b;
  }
  r += "]";
  snprintf(buf, len, "%s", r.c_str());
  return r.size() < len ? ISDF_OK : ISDF_ERR_ARG;
}

int isdf_set_workspace_limit(isdf_handle* h, uint64_t bytes) {
  if (!h) return ISDF_ERR_ARG;
  if (bytes == 0) return fail(h, ISDF_ERR_ARG, "workspace limit must be positive");
  h->split_budget = (size_t)bytes;
  return ISDF_OK;
}

int isdf_get(isdf_handle* h, int what, void* out) {
  if (!h || !out) return ISDF_ERR_ARG;
  LaunchScope ls(h);
  if (int e = check_device(h)) return e;
  const int nk = h->nk, np = h->np, ng = h->ng, nao = h->nao;
  switch (what) {
    case 0:
      if (!h->has_points) return fail(h, ISDF_ERR_STATE, "X not available");
      CK(cudaMemcpyAsync(out, h->buf("X"), sizeof(double2) * (size_t)nk * np * nao, cudaMemcpyDeviceToDevice, h->st));
      break;
    case 1:
      if (!h->has_fit) return fail(h, ISDF_ERR_STATE, "Pi not available");
      CK(cudaMemcpyAsync(out, h->buf("Pi"), sizeof(double2) * (size_t)nk * np * np, cudaMemcpyDeviceToDevice, h->st));
      break;
    case 2:
      if (!h->has_eta) return fail(h, ISDF_ERR_STATE, "eta not available (needs isdf_fit_zeta)");
      CK(cudaMemcpyAsync(out, h->buf("eta"), sizeof(double2) * (size_t)nk * np * ng, cudaMemcpyDeviceToDevice, h->st));
      break;
    case 3: {
      if (!h->has_xi) return fail(h, ISDF_ERR_STATE, "zeta not available (needs isdf_fit_zeta, before the metric)");
      const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
      // zeta = W^H xi with the rx stored rows of xi
      const int rx = h->xi_rows;
      CK(zgemm(h->st, 'C', 'N', np, ng, rx, one, (double2*)h->buf("W"), np, (int64_t)np * np, (double2*)h->buf("xi"),
               ng, (int64_t)rx * ng, zero, (double2*)out, ng, (int64_t)np * ng, nk));
      break;
    }
    default:
      return fail(h, ISDF_ERR_ARG, "unknown item %d", what);
  }
  CK(cudaStreamSynchronize(h->st));
  return ISDF_OK;
}

int isdf_sizes(const isdf_handle* h, int64_t* out) {
  if (!h || !out) return ISDF_ERR_ARG;
  out[0] = h->nao;
  out[1] = h->nk;
  out[2] = h->ng;
  out[3] = h->has_points ? h->np : 0;
  return ISDF_OK;
}

int64_t isdf_launch_count(const isdf_handle* h) { return h ? h->launches : 0; }

int isdf_timing_enable(isdf_handle* h, int enable) {
  if (!h) return ISDF_ERR_ARG;
  if (!h->pending.empty()) {
    cudaStreamSynchronize(h->st);
    h->resolve_timing();
  }
  h->timing = enable != 0;
  if (h->timing)
    for (int i = 0; i < isdf_handle::kStages; ++i) {
      h->stage_ms[i] = 0;
      h->stage_n[i] = 0;
      h->stage_flops[i] = 0;
    }
  return ISDF_OK;
}

int isdf_timing_get(const isdf_handle* h, int stage, double* ms_total, int64_t* launches, double* flops_total) {
  if (!h || stage < 0 || stage >= isdf_handle::kStages) return ISDF_ERR_ARG;
  if (ms_total) *ms_total = h->stage_ms[stage];
  if (launches) *launches = h->stage_n[stage];
  if (flops_total) *flops_total = h->stage_flops[stage];
  return ISDF_OK;
}

const char* isdf_last_error(const isdf_handle* h) { return h ? h->err.c_str() : isdf::noalloc_last_error(); }

void isdf_destroy(isdf_handle* h) {
  if (!h) return;
  if (!h->pending.empty()) cudaStreamSynchronize(h->st);
  for (auto& p : h->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : h->event_pool) cudaEventDestroy(e);
  for (auto& b : h->bufs)
    if (b.second.p) cudaFree(b.second.p);
  delete h;
}

}  // extern "C"
