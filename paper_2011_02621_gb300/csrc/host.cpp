// Host side of the C ABI in include/tn.h: validation, single-qubit fusion and
// gate split (Eq. gatesplit), the two-sided evolution programs with static
// structural bond bounds (Eqs. result1/result2, svd/svd2, shouwei; Fig. 2a),
// Algorithm 1 of the supplement (best-first path search over qubit subsets
// under Assumptions 1-3), cutting, the plan compiler, and the device driver
// of tn_amplitudes.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <queue>
#include <string>
#include <type_traits>
#include <unordered_set>
#include <vector>

#include "tc_persist.h"
#include "tn_host.h"

typedef std::complex<double> cd;

// ---------------------------------------------------------------------------
// errors and launch accounting
// ---------------------------------------------------------------------------
static thread_local std::string g_err;
static std::atomic<int64_t> g_launches{0};

tn_status tn_fail(tn_status s, const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

void tn_count_launch(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

extern "C" int64_t tn_launch_count(int32_t reset) {
  return reset ? g_launches.exchange(0) : g_launches.load();
}

extern "C" const char *tn_last_error(void) { return g_err.c_str(); }

// Runs f (returning tn_status) so that no C++ exception crosses the C ABI: host memory
// exhaustion becomes TN_ERR_OOM, anything else TN_ERR_UNSUPPORTED with its message.
template <typename F>
static tn_status no_throw(const char *what, F &&f) {
  try {
    return f();
  } catch (const std::bad_alloc &) {
    return tn_fail(TN_ERR_OOM, "%s: host memory exhausted", what);
  } catch (const std::exception &e) {
    return tn_fail(TN_ERR_UNSUPPORTED, "%s: %s", what, e.what());
  }
}

// ---------------------------------------------------------------------------
// tracing
// ---------------------------------------------------------------------------
namespace {
struct ProfKind {
  std::string name;
  int64_t launches = 0;
  double ms = 0, bytes = 0, flops = 0;
};
struct ProfRec {
  int kind;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
bool g_prof_steps = false;              // one record per contraction step
thread_local int g_prof_step = -1;      // the contraction step this thread enqueues (-1: none)
std::vector<ProfKind> g_kinds;
std::vector<ProfRec> g_recs;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t prof_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void prof_drain() {   // caller holds the mutex
  for (auto &r : g_recs) {
    float ms = 0;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess)
      g_kinds[r.kind].ms += ms;
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_recs.clear();
  cudaGetLastError();
}
}  // namespace

ProfScope::ProfScope(const char *kind, cudaStream_t stream, double bytes, double flops) {
  if (!g_prof_on) return;
  // no events inside a stream capture (work captured into a graph is timed by its launch)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return;
  std::string name = kind;
  if (g_prof_steps && g_prof_step >= 0) name += "#" + std::to_string(g_prof_step);
  int k = -1;
  for (size_t i = 0; i < g_kinds.size(); ++i)
    if (g_kinds[i].name == name) k = (int)i;
  if (k < 0) {
    g_kinds.push_back(ProfKind());
    g_kinds.back().name = name;
    k = (int)g_kinds.size() - 1;
  }
  g_kinds[k].launches += 1;
  g_kinds[k].bytes += bytes;
  g_kinds[k].flops += flops;
  ProfRec r{k, prof_event(), prof_event()};
  cudaEventRecord(r.a, stream);
  g_recs.push_back(r);
  slot = (int)g_recs.size() - 1;
  st = stream;
}

ProfStep::ProfStep(int step) { g_prof_step = step; }
ProfStep::~ProfStep() { g_prof_step = -1; }

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot < (int)g_recs.size()) cudaEventRecord(g_recs[slot].b, st);
}

extern "C" tn_status tn_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_drain();
  g_kinds.clear();
  g_prof_on = on != 0;
  g_prof_steps = on == 2;
  return TN_OK;
}

extern "C" tn_status tn_profile_read(int32_t idx, char *name, int32_t name_len, int64_t *launches, double *ms,
                                     double *bytes, double *flops) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_drain();
  if (idx < 0 || idx >= (int)g_kinds.size()) return TN_ERR_ARG;
  const ProfKind &k = g_kinds[idx];
  if (name && name_len > 0) {
    std::strncpy(name, k.name.c_str(), name_len - 1);
    name[name_len - 1] = 0;
  }
  if (launches) *launches = k.launches;
  if (ms) *ms = k.ms;
  if (bytes) *bytes = k.bytes;
  if (flops) *flops = k.flops;
  return TN_OK;
}

// ---------------------------------------------------------------------------
// device memory
// ---------------------------------------------------------------------------
void *DevMem::alloc(size_t bytes, cudaStream_t st) {
  if (!bytes) return nullptr;
  if (has) return a.alloc(bytes, (void *)st, a.ctx);
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void DevMem::release(Buf &b) {
  if (!b.p) return;
  if (has) a.free(b.p, b.bytes, (void *)b.stream, a.ctx);
  else cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

tn_status DevMem::ensure(Buf &b, size_t bytes, cudaStream_t st) {
  if (b.p && b.bytes >= bytes) return TN_OK;
  release(b);
  if (!bytes) return TN_OK;
  b.p = alloc(bytes, st);
  if (!b.p) return tn_fail(TN_ERR_OOM, "device allocation of %zu bytes failed", bytes);
  b.bytes = bytes;
  b.stream = st;
  return TN_OK;
}

// ---------------------------------------------------------------------------
// small host SVD (one-sided Jacobi, complex) for the 4x4 gate split
// ---------------------------------------------------------------------------
// X: m x n column-major (n <= m). On return X holds U (unit columns, sorted by
// descending singular value), S the singular values, V (n x n, column-major)
// with X_in = U diag(S) V^H.
static void host_svd(int m, int n, std::vector<cd> &X, std::vector<double> &S, std::vector<cd> &V) {
  V.assign((size_t)n * n, cd(0, 0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rot = false;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double al = 0, be = 0;
        cd ga = 0;
        for (int r = 0; r < m; ++r) {
          cd a = X[(size_t)p * m + r], b = X[(size_t)q * m + r];
          al += std::norm(a);
          be += std::norm(b);
          ga += std::conj(a) * b;
        }
        double g = std::abs(ga);
        if (!(g > 2.0 * std::sqrt((double)m) * 2.220446049250313e-16 * std::sqrt(al * be)) || g == 0.0) continue;
        rot = true;
        double zeta = (be - al) / (2 * g);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1 + zeta * zeta));
        double c = 1 / std::sqrt(1 + t * t), s = c * t;
        cd e = std::conj(ga) / g;
        for (int r = 0; r < m; ++r) {
          cd a = X[(size_t)p * m + r], b = X[(size_t)q * m + r] * e;
          X[(size_t)p * m + r] = c * a - s * b;
          X[(size_t)q * m + r] = s * a + c * b;
        }
        for (int r = 0; r < n; ++r) {
          cd a = V[(size_t)p * n + r], b = V[(size_t)q * n + r] * e;
          V[(size_t)p * n + r] = c * a - s * b;
          V[(size_t)q * n + r] = s * a + c * b;
        }
      }
    if (!rot) break;
  }
  S.assign(n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s2 = 0;
    for (int r = 0; r < m; ++r) s2 += std::norm(X[(size_t)j * m + r]);
    S[j] = std::sqrt(s2);
  }
  std::vector<int> idx(n);
  for (int j = 0; j < n; ++j) idx[j] = j;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return S[a] > S[b]; });
  std::vector<cd> X2((size_t)m * n), V2((size_t)n * n);
  std::vector<double> S2(n);
  for (int t = 0; t < n; ++t) {
    int j = idx[t];
    S2[t] = S[j];
    for (int r = 0; r < m; ++r) X2[(size_t)t * m + r] = S[j] > 0 ? X[(size_t)j * m + r] / S[j] : cd(0, 0);
    for (int r = 0; r < n; ++r) V2[(size_t)t * n + r] = V[(size_t)j * n + r];
  }
  X.swap(X2);
  V.swap(V2);
  S.swap(S2);
}

// Eq. gatesplit on a 4x4 matrix O[(k' l'), (k l)]: P[k'][k][s], Q[l'][l][s].
static int gate_split(const cd *O, cd P[16], cd Q[16]) {
  std::vector<cd> R(16);   // column-major, rows (k'k), cols (l'l)
  for (int kp = 0; kp < 2; ++kp)
    for (int lp = 0; lp < 2; ++lp)
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l) R[(size_t)(lp * 2 + l) * 4 + (kp * 2 + k)] = O[(kp * 2 + lp) * 4 + (k * 2 + l)];
  std::vector<double> S;
  std::vector<cd> V;
  host_svd(4, 4, R, S, V);
  int chi = 0;
  for (int s = 0; s < 4; ++s) chi += (S[s] > 1e-12 * S[0]) ? 1 : 0;
  for (int i = 0; i < 16; ++i) P[i] = Q[i] = 0;
  for (int s = 0; s < chi; ++s) {
    double r = std::sqrt(S[s]);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        P[(a * 2 + b) * 4 + s] = R[(size_t)s * 4 + (a * 2 + b)] * r;
        Q[(a * 2 + b) * 4 + s] = std::conj(V[(size_t)s * 4 + (a * 2 + b)]) * r;
      }
  }
  return chi;
}

extern "C" tn_status tn_gate_split(const tn_c128 *m, tn_c128 *P, tn_c128 *Q, int32_t *chi_o) {
  if (!m || !P || !Q || !chi_o) return tn_fail(TN_ERR_ARG, "tn_gate_split: NULL argument");
  cd O[16], Pc[16], Qc[16];
  for (int i = 0; i < 16; ++i) O[i] = cd(m[i].re, m[i].im);
  *chi_o = gate_split(O, Pc, Qc);
  for (int i = 0; i < 16; ++i) {
    P[i].re = Pc[i].real(); P[i].im = Pc[i].imag();
    Q[i].re = Qc[i].real(); Q[i].im = Qc[i].imag();
  }
  return TN_OK;
}

// ---------------------------------------------------------------------------
// graph checks
// ---------------------------------------------------------------------------
// max_nodes: 128 for qubit graphs of circuits, 256 for the graphs of the host-only path and cut
// searches (Algorithm 1's subset masks hold up to 256 nodes)
static tn_status check_graph(const tn_graph *g, std::vector<int> &eu, std::vector<int> &ev,
                             std::vector<std::vector<int>> &legs, int max_nodes = 128) {
  if (!g || g->n_qubits <= 0 || g->n_edges < 0 || (g->n_edges > 0 && !g->edges))
    return tn_fail(TN_ERR_ARG, "graph: bad sizes or NULL edges");
  const int n = g->n_qubits, ne = g->n_edges;
  if (n > max_nodes) return tn_fail(TN_ERR_UNSUPPORTED, "graph: at most %d nodes are supported (got %d)", max_nodes, n);
  eu.resize(ne);
  ev.resize(ne);
  legs.assign(n, {});
  std::unordered_set<int64_t> seen;
  for (int i = 0; i < ne; ++i) {
    int u = g->edges[2 * i], v = g->edges[2 * i + 1];
    if (u < 0 || v < 0 || u >= n || v >= n) return tn_fail(TN_ERR_GRAPH, "edge %d: endpoint out of range", i);
    if (u == v) return tn_fail(TN_ERR_GRAPH, "edge %d: self loop", i);
    int64_t key = (int64_t)std::min(u, v) * 1024 + std::max(u, v);
    if (!seen.insert(key).second) return tn_fail(TN_ERR_GRAPH, "edge %d: duplicate edge", i);
    eu[i] = u;
    ev[i] = v;
    legs[u].push_back(i);
    legs[v].push_back(i);
  }
  for (int q = 0; q < n; ++q)
    if ((int)legs[q].size() > TN_MAXLEG)
      return tn_fail(TN_ERR_UNSUPPORTED, "qubit %d has degree %zu > %d", q, legs[q].size(), TN_MAXLEG);
  // connectivity
  std::vector<int> comp(n, 0), st{0};
  comp[0] = 1;
  while (!st.empty()) {
    int x = st.back();
    st.pop_back();
    for (int e : legs[x]) {
      int y = eu[e] == x ? ev[e] : eu[e];
      if (!comp[y]) { comp[y] = 1; st.push_back(y); }
    }
  }
  for (int q = 0; q < n; ++q)
    if (!comp[q]) return tn_fail(TN_ERR_GRAPH, "graph is not connected (qubit %d unreachable)", q);
  return TN_OK;
}

static int find_edge(const tn_circuit *c, int a, int b) {
  for (int e : c->legs[a])
    if ((c->eu[e] == a && c->ev[e] == b) || (c->eu[e] == b && c->ev[e] == a)) return e;
  return -1;
}

extern "C" tn_status tn_build(const tn_graph *g, const tn_gate *gates, int64_t n_gates, const tn_allocator *alloc,
                              tn_circuit **out) {
  if (!out) return tn_fail(TN_ERR_ARG, "tn_build: out is NULL");
  *out = nullptr;
  if (n_gates < 0 || (n_gates > 0 && !gates)) return tn_fail(TN_ERR_ARG, "tn_build: bad gate list");
  tn_circuit *c = new tn_circuit();
  tn_status s = check_graph(g, c->eu, c->ev, c->legs);
  if (s != TN_OK) { delete c; return s; }
  c->n = g->n_qubits;
  c->ne = g->n_edges;
  for (int64_t i = 0; i < n_gates; ++i) {
    const tn_gate &gt = gates[i];
    if (gt.arity != 1 && gt.arity != 2) { delete c; return tn_fail(TN_ERR_ARG, "gate %lld: arity %d", (long long)i, gt.arity); }
    if (gt.cycle < 1) { delete c; return tn_fail(TN_ERR_ARG, "gate %lld: cycle must be >= 1", (long long)i); }
    for (int j = 0; j < gt.arity; ++j)
      if (gt.q[j] < 0 || gt.q[j] >= c->n) { delete c; return tn_fail(TN_ERR_GRAPH, "gate %lld: qubit out of range", (long long)i); }
    if (gt.arity == 2 && find_edge(c, gt.q[0], gt.q[1]) < 0) {
      delete c;
      return tn_fail(TN_ERR_GRAPH, "gate %lld acts on (%d,%d), which is not an edge", (long long)i, gt.q[0], gt.q[1]);
    }
    for (int j = 0; j < (gt.arity == 2 ? 16 : 4); ++j)
      if (!std::isfinite(gt.m[j].re) || !std::isfinite(gt.m[j].im)) {
        delete c;
        return tn_fail(TN_ERR_ARG, "gate %lld: non-finite matrix entry", (long long)i);
      }
    c->gates.push_back(gt);
  }
  c->max_deg = 0;
  for (int q = 0; q < c->n; ++q) c->max_deg = std::max(c->max_deg, (int)c->legs[q].size());
  if (alloc) { c->mem.a = *alloc; c->mem.has = alloc->alloc && alloc->free; }
  *out = c;
  return TN_OK;
}

// ---------------------------------------------------------------------------
// evolution programs
// ---------------------------------------------------------------------------
typedef std::array<cd, 4> M2;

static M2 mul2(const M2 &a, const M2 &b) {
  M2 r;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) r[i * 2 + j] = a[i * 2] * b[j] + a[i * 2 + 1] * b[2 + j];
  return r;
}

// Build one half: `seq` in processing order, matrices transposed for the bra.
// Single-qubit gates accumulate per qubit and fuse into the next two-qubit
// gate on that qubit (its input side); leftovers become tail applications.
// caps / cap_sv (optional): probed rank per two-qubit step and the endpoint it was probed on;
// a cap applies only where this program SVDs the same endpoint.
// The half's gate program with static shapes. Without `force_sv` every compression SVDs the
// endpoint with fewer rows 2 * prod(other legs) (ties: q[0]) and the bond becomes
// min(dim * chi_o, those rows, chi): the structural program, independent of the state. With
// `force_sv` (the structural program's endpoints) and `caps` (probed ranks), the same endpoints
// are kept and each bond is also capped by its probed rank. With the two-sided compression every
// two-qubit gate is two entries (see below); force_sv and caps are per entry.
static void build_half(const tn_circuit *c, const std::vector<const tn_gate *> &seq, bool transpose, int chi,
                       double cutoff, Half &h, const std::vector<int> *caps = nullptr,
                       const std::vector<int> *force_sv = nullptr) {
  const int n = c->n;
  const bool two_sided = c->compress == TN_COMPRESS_TWO_SIDED;
  h = Half();
  h.max_sweeps = c->max_sweeps;
  h.dims.assign(c->ne, 1);
  std::vector<M2> pend(n, M2{1, 0, 0, 1});
  std::vector<char> has(n, 0);
  std::vector<int64_t> cap(n, 2);
  auto node_size = [&](int q) {
    int64_t s = 2;
    for (int e : c->legs[q]) s *= h.dims[e];
    return s;
  };
  for (const tn_gate *g : seq) {
    if (g->arity == 1) {
      M2 u;
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          const tn_c128 &x = transpose ? g->m[j * 2 + i] : g->m[i * 2 + j];
          u[i * 2 + j] = cd(x.re, x.im);
        }
      pend[g->q[0]] = mul2(u, pend[g->q[0]]);
      has[g->q[0]] = 1;
      continue;
    }
    const int k = g->q[0], l = g->q[1];
    cd O[16], F[16];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const tn_c128 &x = transpose ? g->m[j * 4 + i] : g->m[i * 4 + j];
        O[i * 4 + j] = cd(x.re, x.im);
      }
    // F = O (pend_k (x) pend_l), basis |k l>, k the high bit
    const M2 &pk = pend[k], &pl = pend[l];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        cd acc = 0;
        for (int t = 0; t < 4; ++t) acc += O[i * 4 + t] * pk[(t >> 1) * 2 + (j >> 1)] * pl[(t & 1) * 2 + (j & 1)];
        F[i * 4 + j] = acc;
      }
    pend[k] = pend[l] = M2{1, 0, 0, 1};
    has[k] = has[l] = 0;
    cd P[16], Q[16];
    int chi_o = gate_split(F, P, Q);
    const int e = find_edge(c, k, l);
    // One entry of the program: gate (Pm, Qm) with chi_o_ terms on (k, l) at the current bonds,
    // SVD of endpoint k (sv_rule 1) or l (0) unless force_sv names it, bond bound dout (capped
    // by chi unless `whole`, and by the probed rank), keep rule s_j > cut * s_0.
    auto entry = [&](const cd *Pm, const cd *Qm, int chi_o_, int sv_rule, bool whole, double cut) {
      GateParams gp;
      std::memset(&gp, 0, sizeof gp);
      gp.nk = (int)c->legs[k].size();
      gp.nl = (int)c->legs[l].size();
      int64_t ok = 1, ol = 1;
      for (int j = 0; j < gp.nk; ++j) {
        int ej = c->legs[k][j];
        gp.dk[j] = h.dims[ej];
        if (ej == e) gp.pk = j; else ok *= h.dims[ej];
      }
      for (int j = 0; j < gp.nl; ++j) {
        int ej = c->legs[l][j];
        gp.dl[j] = h.dims[ej];
        if (ej == e) gp.pl = j; else ol *= h.dims[ej];
      }
      gp.din = h.dims[e];
      gp.chi_o = chi_o_;
      gp.n = gp.din * chi_o_;
      gp.m_k = (int)(2 * ok);
      gp.m_l = (int)(2 * ol);
      const size_t gi = h.gp.size();
      gp.sv_is_k = sv_rule;
      if (force_sv && gi < force_sv->size()) gp.sv_is_k = (*force_sv)[gi];
      int dout = std::min(gp.n, gp.sv_is_k ? gp.m_k : gp.m_l);
      if (chi > 0 && !whole) dout = std::min(dout, chi);
      if (caps && gi < caps->size() && (*caps)[gi] > 0) dout = std::min(dout, (*caps)[gi]);   // probed rank
      gp.dout = dout;
      gp.id = (int)gi;
      gp.cutoff = cut;
      for (int i = 0; i < 16; ++i) {
        gp.P[i] = make_double2(Pm[i].real(), Pm[i].imag());
        gp.Q[i] = make_double2(Qm[i].real(), Qm[i].imag());
      }
      h.dims[e] = dout;
      cap[k] = std::max(cap[k], node_size(k));
      cap[l] = std::max(cap[l], node_size(l));
      h.gp.push_back(gp);
      h.gate_nodes.push_back({k, l});
      h.seq.push_back({2, (int)h.gp.size() - 1});
      h.max_gate_mn = std::max<int64_t>(h.max_gate_mn, (int64_t)std::max(gp.m_k, gp.m_l) * gp.n);
    };
    // the endpoint with fewer rows 2 * prod(other legs) is compressed (ties: q[0]); the other
    // legs' dims do not change within one gate
    int64_t rows_k = 2, rows_l = 2;
    for (int ej : c->legs[k]) if (ej != e) rows_k *= h.dims[ej];
    for (int ej : c->legs[l]) if (ej != e) rows_l *= h.dims[ej];
    const int sv = rows_k <= rows_l ? 1 : 0;
    if (!two_sided) {
      entry(P, Q, chi_o, sv, false, cutoff);
      continue;
    }
    // Two-sided: first the gate with the other endpoint decomposed whole (cutoff 0, no chi cap),
    // which leaves that endpoint an isometry U_o and moves S_o V_o^H into A^sv; then an identity
    // gate (one term) decomposing A^sv with the keep rule. A^sv A^o^T = A^sv' U_o^T with U_o's
    // columns orthonormal, so the second SVD has the singular values of the local product.
    const size_t gi = h.gp.size();
    const int sv2 = (force_sv && gi + 1 < force_sv->size()) ? (*force_sv)[gi + 1] : sv;
    entry(P, Q, chi_o, 1 - sv2, true, 0.0);
    cd I[16];
    for (int i = 0; i < 16; ++i) I[i] = 0;
    I[(0 * 2 + 0) * 4 + 0] = 1;     // [s'][s][a]: delta(s', s), one term
    I[(1 * 2 + 1) * 4 + 0] = 1;
    entry(I, I, 1, sv2, false, cutoff);
  }
  for (int q = 0; q < n; ++q) {
    if (!has[q]) continue;
    Apply1Params a;
    std::memset(&a, 0, sizeof a);
    for (int i = 0; i < 4; ++i) a.u[i] = make_double2(pend[q][i].real(), pend[q][i].imag());
    a.size_rest = node_size(q) / 2;
    h.ap.push_back(a);
    h.ap_node.push_back(q);
    h.seq.push_back({1, (int)h.ap.size() - 1});
  }
  // node slots
  h.node_off.assign(n, 0);
  int64_t off = 0;
  for (int q = 0; q < n; ++q) {
    h.node_off[q] = off;
    off += (cap[q] + 1) & ~1LL;      // keep 32-byte alignment of double2 slots
  }
  h.item_elems = std::max<int64_t>(off, 2);
  h.max_work = 0;
  for (size_t i = 0; i < h.gp.size(); ++i) {
    GateParams &gp = h.gp[i];
    gp.off_k = h.node_off[h.gate_nodes[i].first];
    gp.off_l = h.node_off[h.gate_nodes[i].second];
    int64_t w = gate_work_elems(gp);
    gp.use_smem = (w * (int64_t)sizeof(double2) <= 200 * 1024) ? 1 : 0;
    gp.work_stride = w;
    if (!gp.use_smem) h.max_work = std::max(h.max_work, w);
  }
  for (size_t i = 0; i < h.ap.size(); ++i) h.ap[i].off = h.node_off[h.ap_node[i]];
}

static double gate_bytes(const GateParams &g) {   // node tensors in and out (complex128)
  double in = (double)g.m_k / 2 * g.din * 2 + (double)g.m_l / 2 * g.din * 2;
  double out = (double)g.m_k / 2 * g.dout * 2 + (double)g.m_l / 2 * g.dout * 2;
  return 16.0 * (in + out);
}

static double gate_flops(const GateParams &g) {
  // complex gate application (2 terms per element) + one-sided Jacobi thin SVD of an m x n
  // matrix (Golub & Van Loan's count for the one-sided Jacobi method, ~ 2 m n^2 per sweep,
  // 6 sweeps, complex = 4x real) + absorption GEMM
  const double m = g.sv_is_k ? g.m_k : g.m_l, mo = g.sv_is_k ? g.m_l : g.m_k;
  const double r = std::max(m, (double)g.n), c = std::min(m, (double)g.n);
  return 8.0 * 2 * (g.m_k + g.m_l) * g.n + 4.0 * 6 * 2 * r * c * c + 8.0 * mo * g.n * g.dout;
}

tn_status run_half(const Half &h, int n_qubits, double2 *base, int items, const int64_t *node_off_dev,
                   const uint64_t *bits_dev, int words, double2 *gwork, int *errflag, cudaStream_t st,
                   int *rank_out_dev, const double2 *init_vec_dev, int64_t item_stride) {
  const int64_t stride = item_stride > 0 ? item_stride : h.item_elems;
  {
    ProfScope ps("init_product", st, 32.0 * items * n_qubits, 0);
    CUDA_TRY(launch_init_product(base, stride, items, node_off_dev, n_qubits, bits_dev, words, init_vec_dev, st));
  }
  for (const auto &op : h.seq) {
    if (op.first == 2) {
      GateParams g = h.gp[op.second];
      g.max_sweeps = h.max_sweeps;
      ProfScope ps("gate_svd_fp64", st, gate_bytes(g) * items, gate_flops(g) * items);
      CUDA_TRY(launch_gate(g, base, stride, items, gwork, errflag, rank_out_dev ? rank_out_dev + op.second : nullptr,
                           st));
    } else {
      const Apply1Params &a = h.ap[op.second];
      ProfScope ps("apply_1q_fp64", st, 64.0 * a.size_rest * items, 16.0 * a.size_rest * items);
      CUDA_TRY(launch_apply1(a, base, stride, items, st));
    }
  }
  return TN_OK;
}

static tn_status init_device(int &dev) {
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) {
    cudaGetLastError();
    return tn_fail(TN_ERR_CUDA, "no CUDA device available: this library has no CPU fallback");
  }
  CUDA_TRY(cudaGetDevice(&dev));
  return TN_OK;
}

// Run one half once (one item) and read back the numerical rank of every compression.
// `init` = per-qubit 2-vectors of a product initial state (NULL: |0...0>).
static tn_status probe_ranks(tn_circuit *c, const Half &h, const std::vector<double2> *init, std::vector<int> &caps,
                             cudaStream_t st) {
  DevMem &mem = c->mem;
  Buf region, offs, work, ranks, ivec, err;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    mem.release(region);
    mem.release(offs);
    mem.release(work);
    mem.release(ranks);
    mem.release(ivec);
    mem.release(err);
  };
  const size_t ng = std::max<size_t>(h.gp.size(), 1);
  tn_status s;
  if ((s = mem.ensure(region, h.item_elems * sizeof(double2), st)) != TN_OK ||
      (s = mem.ensure(offs, c->n * sizeof(int64_t), st)) != TN_OK ||
      (s = mem.ensure(work, std::max<int64_t>(h.max_work, 1) * sizeof(double2), st)) != TN_OK ||
      (s = mem.ensure(ranks, ng * sizeof(int), st)) != TN_OK ||
      (s = mem.ensure(ivec, 2 * c->n * sizeof(double2), st)) != TN_OK || (s = mem.ensure(err, 16, st)) != TN_OK) {
    cleanup();
    return s;
  }
  cudaError_t e = cudaMemcpyAsync(offs.p, h.node_off.data(), c->n * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && init)
    e = cudaMemcpyAsync(ivec.p, init->data(), 2 * c->n * sizeof(double2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ranks.p, 0, ng * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err.p, 0, 16, st);
  if (e != cudaSuccess) {
    cleanup();
    return tn_fail(TN_ERR_CUDA, "rank probe set-up: %s", cudaGetErrorString(e));
  }
  s = run_half(h, c->n, (double2 *)region.p, 1, (const int64_t *)offs.p, nullptr, 1, (double2 *)work.p,
               (int *)err.p, st, (int *)ranks.p, init ? (const double2 *)ivec.p : nullptr);
  if (s != TN_OK) {
    cleanup();
    return s;
  }
  caps.assign(h.gp.size(), 0);
  int errv = 0;
  e = cudaMemcpyAsync(caps.data(), ranks.p, h.gp.size() * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&errv, err.p, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return tn_fail(TN_ERR_CUDA, "rank probe: %s", cudaGetErrorString(e));
  if (errv) {
    const GateParams &g = h.gp[std::min<size_t>(errv - 1, h.gp.size() - 1)];
    return tn_fail(TN_ERR_TIMEOUT,
                   "Jacobi SVD did not converge within its sweep limit (rank probe, gate %d: m_k %d m_l %d n %d "
                   "din %d dout %d svd %s)",
                   errv - 1, g.m_k, g.m_l, g.n, g.din, g.dout, g.sv_is_k ? "k" : "l");
  }
  for (int &x : caps) x = std::max(x, 1);
  return TN_OK;
}

extern "C" tn_status tn_evolve_two_sided(tn_circuit *c, int32_t split_cycle, int32_t chi_max, double cutoff_rel,
                                         void *cuda_stream) {
  if (!c) return tn_fail(TN_ERR_ARG, "tn_evolve_two_sided: NULL circuit");
  if (split_cycle < 0 || chi_max < 0 || !(cutoff_rel >= 0) || cutoff_rel >= 1)
    return tn_fail(TN_ERR_ARG, "tn_evolve_two_sided: bad split/chi/cutoff");
  tn_status s = init_device(c->device);
  if (s != TN_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the same program again keeps plans valid (same static shapes); anything else rebuilds it
  const bool same = c->evolved && c->split == split_cycle && c->chi == chi_max && c->cutoff == cutoff_rel &&
                    c->built_compress == c->compress;
  DevMem &mem = c->mem;
  if (!same) {
    std::vector<const tn_gate *> g1, g2;
    for (const auto &g : c->gates) (g.cycle <= split_cycle ? g1 : g2).push_back(&g);
    std::reverse(g2.begin(), g2.end());
    build_half(c, g1, false, chi_max, cutoff_rel, c->ket);
    build_half(c, g2, true, chi_max, cutoff_rel, c->bra);
    c->split = split_cycle;
    c->chi = chi_max;
    c->cutoff = cutoff_rel;
    c->built_compress = c->compress;
    // Rank probe. The static bounds can exceed the true bond ranks. The ket is a single state:
    // its ranks are exact. For the bra, the ranks reached from one random (generic) product state
    // bound those reached from every basis state (a rank can only drop on special inputs), so
    // they are safe static shapes; rank deficits stay zero-padded. Every rebuilt program SVDs the
    // structural program's endpoints (which endpoint is compressed changes a truncated result, so
    // it must not depend on the data), capped by the probed ranks, and is probed again until the
    // shapes stop shrinking (at most four rounds).
    c->evolved = false;
    std::vector<double2> gen_init(2 * c->n);
    {
      uint64_t x = 0x9E3779B97F4A7C15ull;   // fixed splitmix64 stream: deterministic shapes
      auto u = [&x]() {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
      };
      for (auto &v : gen_init) v = make_double2(u(), u());
    }
    for (int side = 0; side < 2; ++side) {
      const std::vector<const tn_gate *> &seq = side == 0 ? g1 : g2;
      Half &h = side == 0 ? c->ket : c->bra;
      std::vector<int> sv(h.gp.size());     // the structural program's endpoints, kept throughout
      for (size_t i = 0; i < h.gp.size(); ++i) sv[i] = h.gp[i].sv_is_k;
      for (int round = 0; round < 4; ++round) {
        std::vector<int> caps;
        tn_status ps = probe_ranks(c, h, side == 0 ? nullptr : &gen_init, caps, st);
        if (ps != TN_OK) return ps;
        Half next;
        build_half(c, seq, side == 1, chi_max, cutoff_rel, next, &caps, &sv);
        const bool changed = next.dims != h.dims || next.item_elems != h.item_elems;
        h = next;
        if (!changed) break;
      }
    }
  }
  c->evolved = false;
  // upload node offsets, run the ket half (one item)
  if ((s = mem.ensure(c->ket_dev, c->ket.item_elems * sizeof(double2), st)) != TN_OK) return s;
  if ((s = mem.ensure(c->ket_c64, c->ket.item_elems * sizeof(float2), st)) != TN_OK) return s;
  if ((s = mem.ensure(c->ket_off_dev, c->n * sizeof(int64_t), st)) != TN_OK) return s;
  if ((s = mem.ensure(c->bra_off_dev, c->n * sizeof(int64_t), st)) != TN_OK) return s;
  if ((s = mem.ensure(c->err_dev, sizeof(int), st)) != TN_OK) return s;
  if ((s = mem.ensure(c->ket_work, std::max<int64_t>(c->ket.max_work, 1) * sizeof(double2), st)) != TN_OK) return s;
  CUDA_TRY(cudaMemcpyAsync(c->ket_off_dev.p, c->ket.node_off.data(), c->n * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(c->bra_off_dev.p, c->bra.node_off.data(), c->n * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemsetAsync(c->ket_dev.p, 0, c->ket.item_elems * sizeof(double2), st));
  CUDA_TRY(cudaMemsetAsync(c->err_dev.p, 0, sizeof(int), st));
  s = run_half(c->ket, c->n, (double2 *)c->ket_dev.p, 1, (const int64_t *)c->ket_off_dev.p, nullptr, 1,
               (double2 *)c->ket_work.p, (int *)c->err_dev.p, st, nullptr, nullptr);
  if (s != TN_OK) return s;
  CUDA_TRY(launch_to_c64((const double2 *)c->ket_dev.p, (float2 *)c->ket_c64.p, c->ket.item_elems, st));
  int err = 0;
  CUDA_TRY(cudaMemcpyAsync(&err, c->err_dev.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (err) return tn_fail(TN_ERR_TIMEOUT, "Jacobi SVD did not converge within its sweep limit (ket half, gate %d)", err - 1);
  c->evolved = true;
  if (!same) c->generation++;
  return TN_OK;
}

extern "C" tn_status tn_circuit_bond_dims(const tn_circuit *c, int32_t side, int32_t *out) {
  if (!c || !out || (side != 0 && side != 1)) return tn_fail(TN_ERR_ARG, "tn_circuit_bond_dims: bad argument");
  if (!c->evolved) return tn_fail(TN_ERR_STATE, "tn_circuit_bond_dims: call tn_evolve_two_sided first");
  const Half &h = side == 0 ? c->ket : c->bra;
  for (int e = 0; e < c->ne; ++e) out[e] = h.dims[e];
  return TN_OK;
}

extern "C" void tn_circuit_free(tn_circuit *c) {
  if (!c) return;
  c->mem.release(c->ket_dev);
  c->mem.release(c->ket_c64);
  c->mem.release(c->ket_off_dev);
  c->mem.release(c->bra_off_dev);
  c->mem.release(c->err_dev);
  c->mem.release(c->ket_work);
  delete c;
}

// ---------------------------------------------------------------------------
// Algorithm 1 (supplement): best-first search over qubit subsets
// ---------------------------------------------------------------------------
namespace {
// Node subsets of Algorithm 1 as bit masks of W words: W = 2 for networks of up to 128 nodes,
// W = 4 (with 16-bit node indices in the states) for up to 256, e.g. the double-layer network of
// a 104-qubit circuit. The search itself does not depend on W.
template <int W> struct MaskT {
  uint64_t w[W] = {};
  bool get(int i) const { return (w[i >> 6] >> (i & 63)) & 1; }
  void set(int i) { w[i >> 6] |= 1ull << (i & 63); }
  void clear(int i) { w[i >> 6] &= ~(1ull << (i & 63)); }
  bool operator==(const MaskT &o) const {
    for (int j = 0; j < W; ++j)
      if (w[j] != o.w[j]) return false;
    return true;
  }
  bool any_and(const MaskT &o) const {
    for (int j = 0; j < W; ++j)
      if (w[j] & o.w[j]) return true;
    return false;
  }
};
template <int W> struct MaskHashT {
  size_t operator()(const MaskT<W> &m) const {
    uint64_t h = m.w[0] * 0x9E3779B97F4A7C15ull ^ (m.w[1] + 0x632BE59BD9B4E019ull + (m.w[0] << 6));
    for (int j = 2; j < W; ++j) h = (h ^ m.w[j]) * 0x9E3779B97F4A7C15ull + (h >> 17);
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    return (size_t)(h ^ (h >> 29));
  }
};
template <int W> struct PEntryT {
  using Node = typename std::conditional<W == 2, uint8_t, uint16_t>::type;    // node index / count
  using Iso = typename std::conditional<W == 2, int8_t, int16_t>::type;       // isolated node, -1: none
  MaskT<W> mask;
  double score, prod_open;
  int32_t parent;
  Node last, m;
  uint8_t rank;
  Iso c;
};
struct HeapKey {
  double score;
  int m;
  int64_t seq;
  int32_t idx;
  bool operator<(const HeapKey &o) const {   // priority_queue: "less" = lower priority
    if (score != o.score) return score > o.score;
    if (m != o.m) return m < o.m;
    return seq > o.seq;
  }
};
}  // namespace

struct PathGraph {
  int n;
  std::vector<std::vector<std::pair<int, int>>> adj;   // (neighbour, edge)
  std::vector<double> dims;
};

static PathGraph make_pg(int n, const std::vector<int> &eu, const std::vector<int> &ev, const std::vector<double> &dims) {
  PathGraph pg;
  pg.n = n;
  pg.adj.assign(n, {});
  pg.dims = dims;
  for (size_t e = 0; e < eu.size(); ++e) {
    pg.adj[eu[e]].push_back({ev[e], (int)e});
    pg.adj[ev[e]].push_back({eu[e], (int)e});
  }
  return pg;
}

template <int W>
static tn_status alg1_masks(const PathGraph &pg, int max_rank, bool boundary_only, bool connected,
                            int64_t max_states, std::vector<int> &order, double &score, int64_t &pops,
                            double byte_weight) {
  using Mask = MaskT<W>;
  using PEntry = PEntryT<W>;
  using Node = typename PEntry::Node;
  using Iso = typename PEntry::Iso;
  const int n = pg.n;
  std::vector<Mask> nb(n);                             // neighbour masks
  for (int q = 0; q < n; ++q)
    for (auto &pr : pg.adj[q]) nb[q].set(pr.first);
  std::vector<PEntry> arena;
  arena.reserve(1 << 16);
  std::priority_queue<HeapKey> pq;
  int64_t seq = 0;
  const int64_t arena_cap = std::max<int64_t>(8 * max_states, 1 << 20);
  int maxdeg = 0;
  for (int q = 0; q < n; ++q) maxdeg = std::max(maxdeg, (int)pg.adj[q].size());
  std::vector<int> starts;
  for (int q = 0; q < n; ++q)
    if (!boundary_only || (int)pg.adj[q].size() < maxdeg) starts.push_back(q);
  if (starts.empty())
    for (int q = 0; q < n; ++q) starts.push_back(q);
  for (int q : starts) {
    PEntry e;
    e.mask.set(q);
    e.score = 0;
    double po = 1;
    int rk = 0;
    for (auto &pr : pg.adj[q]) { po *= pg.dims[pr.second]; rk += pg.dims[pr.second] > 1 ? 1 : 0; }
    e.prod_open = po;
    e.parent = -1;
    e.last = (Node)q;
    e.m = 1;
    e.rank = (uint8_t)rk;
    e.c = -1;
    arena.push_back(e);
    pq.push({0.0, 1, seq++, (int32_t)arena.size() - 1});
  }
  std::unordered_set<Mask, MaskHashT<W>> seen;
  pops = 0;
  while (!pq.empty()) {
    HeapKey hk = pq.top();
    pq.pop();
    const PEntry cur = arena[hk.idx];
    if (seen.count(cur.mask)) continue;
    seen.insert(cur.mask);
    if (++pops > max_states) return tn_fail(TN_ERR_NO_PATH, "Algorithm 1: more than %lld states", (long long)max_states);
    if (cur.m == n) {
      order.assign(n, -1);
      int idx = hk.idx, pos = n - 1;
      while (idx >= 0) { order[pos--] = arena[idx].last; idx = arena[idx].parent; }
      score = cur.score;
      return TN_OK;
    }
    // members other than the isolated qubit
    Mask main = cur.mask;
    if (cur.c >= 0) main.clear(cur.c);
    // The nodes the loop below can accept, in ascending order as before: without Assumption 3
    // every non-member; with it the neighbours of the set (of the isolated node when there is
    // one) and, when there is none, the non-members two steps away.
    Mask cand;
    if (!connected) {
      for (int i = 0; i < n; ++i)
        if (!cur.mask.get(i)) cand.set(i);
    } else if (cur.c >= 0) {
      cand = nb[cur.c];
    } else {
      Mask front;
      for (int j = 0; j < W; ++j)
        for (uint64_t b = cur.mask.w[j]; b; b &= b - 1) {
          const Mask &m = nb[j * 64 + __builtin_ctzll(b)];
          for (int t = 0; t < W; ++t) front.w[t] |= m.w[t];
        }
      cand = front;
      for (int j = 0; j < W; ++j)
        for (uint64_t b = front.w[j] & ~cur.mask.w[j]; b; b &= b - 1) {
          const Mask &m = nb[j * 64 + __builtin_ctzll(b)];
          for (int t = 0; t < W; ++t) cand.w[t] |= m.w[t];
        }
    }
    for (int t = 0; t < W; ++t) cand.w[t] &= ~cur.mask.w[t];
    for (int wi = 0; wi < W; ++wi) {
      for (uint64_t bits = cand.w[wi]; bits; bits &= bits - 1) {
        const int i = wi * 64 + __builtin_ctzll(bits);
        const bool adj_s = nb[i].any_and(cur.mask);
        Iso c_new = -1;
        if (connected) {
          if (cur.c >= 0) {
            if (!nb[i].get(cur.c) || !nb[i].any_and(main)) continue;   // must reconnect the isolated qubit
          } else if (!adj_s) {
            bool dist2 = false;            // an isolated qubit must be reconnectable by the next step
            for (auto &pr : pg.adj[i])
              if (nb[pr.first].any_and(cur.mask)) { dist2 = true; break; }
            if (!dist2) continue;
            c_new = (Iso)i;
          }
        }
        double shared = 1, fresh = 1;
        int rk = cur.rank;
        for (auto &pr : pg.adj[i]) {
          const double d = pg.dims[pr.second];
          if (cur.mask.get(pr.first)) { shared *= d; rk -= d > 1 ? 1 : 0; }
          else { fresh *= d; rk += d > 1 ? 1 : 0; }
        }
        if (max_rank > 0 && rk > max_rank) continue;
        PEntry e;
        e.mask = cur.mask;
        e.mask.set(i);
        e.prod_open = cur.prod_open / shared * fresh;
        // Cost = prod of dims over legs of C^S and C^i (+ byte_weight x the step's input and output)
        e.score = cur.score + cur.prod_open * fresh + (byte_weight > 0 ? byte_weight * (cur.prod_open + e.prod_open) : 0.0);
        e.parent = hk.idx;
        e.last = (Node)i;
        e.m = (Node)(cur.m + 1);
        e.rank = (uint8_t)std::max(rk, 0);
        e.c = c_new;
        if ((int64_t)arena.size() >= arena_cap)
          return tn_fail(TN_ERR_NO_PATH, "Algorithm 1: state arena exceeded %lld entries", (long long)arena_cap);
        arena.push_back(e);
        pq.push({e.score, (int)e.m, seq++, (int32_t)arena.size() - 1});
      }
    }
  }
  return tn_fail(TN_ERR_NO_PATH, "Algorithm 1: no path satisfies the assumptions (max_rank %d)", max_rank);
}

static tn_status alg1(const PathGraph &pg, int max_rank, bool boundary_only, bool connected, int64_t max_states,
                      std::vector<int> &order, double &score, int64_t &pops, double byte_weight = 0) {
  if (pg.n <= 128)
    return alg1_masks<2>(pg, max_rank, boundary_only, connected, max_states, order, score, pops, byte_weight);
  if (pg.n <= 256)
    return alg1_masks<4>(pg, max_rank, boundary_only, connected, max_states, order, score, pops, byte_weight);
  return tn_fail(TN_ERR_UNSUPPORTED, "Algorithm 1: at most 256 network nodes (got %d)", pg.n);
}

static tn_status path_auto(const PathGraph &pg, const tn_path_opts &o, std::vector<int> &order, double &score,
                           int64_t &pops, int &rank_used) {
  const int64_t cap = o.max_states > 0 ? o.max_states : 4000000;
  if (o.max_rank > 0 || !o.connected) {
    rank_used = o.max_rank;
    return alg1(pg, o.max_rank, o.boundary_only != 0, o.connected != 0, cap, order, score, pops, o.byte_weight);
  }
  int maxdeg = 0;
  for (int q = 0; q < pg.n; ++q) maxdeg = std::max(maxdeg, (int)pg.adj[q].size());
  // smallest feasible M, then up to three larger ones (a looser rank bound can only lower the
  // score); the lowest score wins
  int64_t total = 0;
  tn_status s = TN_ERR_NO_PATH;
  int first = -1;
  double best = 0;
  std::vector<int> best_order;
  for (int M = std::max(maxdeg, 1); M <= pg.n + 1; ++M) {
    if (first >= 0 && M > first + 3) break;
    int64_t p = 0;
    std::vector<int> ord;
    double sc = 0;
    tn_status r = alg1(pg, M, o.boundary_only != 0, true, cap, ord, sc, p, o.byte_weight);
    total += p;
    if (r != TN_OK) {
      if (first >= 0) break;   // a larger M ran out of states: keep what was found
      continue;
    }
    if (first < 0) first = M;
    if (best_order.empty() || sc < best) {
      best = sc;
      best_order = ord;
      rank_used = M;
    }
    s = TN_OK;
  }
  pops = total;
  if (s == TN_OK) {
    order = best_order;
    score = best;
  }
  return s;
}

static tn_status tn_path_search_impl(const tn_graph *g, const double *dims, const tn_path_opts *opts, int32_t *order,
                                    double *score, int64_t *states_expanded) {
  if (!g || !dims || !order) return tn_fail(TN_ERR_ARG, "tn_path_search: NULL argument");
  std::vector<int> eu, ev;
  std::vector<std::vector<int>> legs;
  tn_status s = check_graph(g, eu, ev, legs, 256);
  if (s != TN_OK) return s;
  std::vector<double> d(dims, dims + g->n_edges);
  for (double x : d)
    if (!(x >= 1)) return tn_fail(TN_ERR_ARG, "tn_path_search: dims must be >= 1");
  tn_path_opts o = tn_default_opts();
  if (opts) o = *opts;
  PathGraph pg = make_pg(g->n_qubits, eu, ev, d);
  std::vector<int> ord;
  double sc = 0;
  int64_t pops = 0;
  int ru = 0;
  s = path_auto(pg, o, ord, sc, pops, ru);
  if (states_expanded) *states_expanded = pops;
  if (s != TN_OK) return s;
  for (int i = 0; i < g->n_qubits; ++i) order[i] = ord[i];
  if (score) *score = sc;
  return TN_OK;
}

extern "C" tn_status tn_path_search(const tn_graph *g, const double *dims, const tn_path_opts *opts, int32_t *order,
                                      double *score, int64_t *states_expanded) {
  return no_throw("tn_path_search", [&] { return tn_path_search_impl(g, dims, opts, order, score, states_expanded); });
}

tn_path_opts tn_default_opts() {
  tn_path_opts o;
  std::memset(&o, 0, sizeof o);
  o.max_rank = 0;
  o.boundary_only = 1;
  o.connected = 1;
  o.max_states = 0;
  o.n_cuts = -1;
  o.max_intermediate = 0;
  o.mem_budget_bytes = 0;
  return o;
}

// ---------------------------------------------------------------------------
// cuts and the plan compiler
// ---------------------------------------------------------------------------
// sizes of the intermediates along `order` (elements), with per-edge dims
static std::vector<double> frontier_sizes(const Net &c, const std::vector<int> &order,
                                          const std::vector<double> &dims, std::vector<std::vector<int>> *open_out) {
  std::vector<char> in(c.n, 0);
  std::vector<double> sizes;
  std::vector<char> open(c.ne, 0);
  for (size_t j = 0; j < order.size(); ++j) {
    int i = order[j];
    in[i] = 1;
    for (int e : c.legs[i]) open[e] = !open[e] ? 1 : 0;   // toggles: opened by first endpoint, closed by second
    double s = 1;
    std::vector<int> op;
    for (int e = 0; e < c.ne; ++e)
      if (open[e]) { s *= dims[e]; op.push_back(e); }
    sizes.push_back(s);
    if (open_out) open_out->push_back(op);
  }
  return sizes;
}

// Cutting (overlap paragraph; positions "where the lattice is the thinnest", supplement):
// greedily cut, among the open legs of the widest intermediate of the current path, the edge
// whose cut network has the smallest total cost (slices x Algorithm 1 score of the cut
// network), until every intermediate fits `limit` (or `want` cuts are made). Returns the
// final path of the cut network.
static tn_status choose_cuts(const Net &c, const tn_path_opts &o, std::vector<double> dims, int want,
                             double limit, std::vector<int> &cuts, std::vector<int> &order, double &score,
                             int64_t &pops, int &rank_used) {
  cuts.clear();
  double slices = 1;
  for (int it = 0; it < c.ne; ++it) {
    std::vector<std::vector<int>> open;
    std::vector<double> sz = frontier_sizes(c, order, dims, &open);
    const double mx = *std::max_element(sz.begin(), sz.end());
    if (want >= 0 ? (int)cuts.size() >= want : mx <= limit) return TN_OK;
    const size_t arg = std::max_element(sz.begin(), sz.end()) - sz.begin();
    int best = -1;
    double best_cost = 0, best_max = 0;
    std::vector<int> best_order;
    int best_rank = 0;
    for (int e : open[arg]) {
      if (dims[e] <= 1) continue;
      std::vector<double> d2 = dims;
      d2[e] = 1;
      PathGraph pg = make_pg(c.n, c.eu, c.ev, d2);
      std::vector<int> ord;
      double sc = 0;
      int64_t pp = 0;
      int ru = 0;
      if (path_auto(pg, o, ord, sc, pp, ru) != TN_OK) continue;
      pops += pp;
      std::vector<double> sz2 = frontier_sizes(c, ord, d2, nullptr);
      const double mx2 = *std::max_element(sz2.begin(), sz2.end());
      const double cost = slices * dims[e] * sc;
      if (best < 0 || cost < best_cost || (cost == best_cost && mx2 < best_max)) {
        best = e; best_cost = cost; best_max = mx2; best_order = ord; best_rank = ru;
      }
    }
    if (best < 0) return want >= 0 ? TN_OK : tn_fail(TN_ERR_NO_PATH, "cutting cannot reach the intermediate limit");
    slices *= dims[best];
    dims[best] = 1;
    cuts.push_back(best);
    order = best_order;
    score = best_cost / slices;
    rank_used = best_rank;
  }
  return TN_OK;
}

static tn_status tn_cut_search_impl(const tn_graph *g, const double *dims, const tn_path_opts *opts, int32_t *order,
                                   int32_t *cuts, int32_t *n_cuts, double *total_cmacs) {
  if (!g || !dims || !order || !n_cuts) return tn_fail(TN_ERR_ARG, "tn_cut_search: NULL argument");
  Net tmp;
  tn_status s = check_graph(g, tmp.eu, tmp.ev, tmp.legs, 256);
  if (s != TN_OK) return s;
  tmp.n = g->n_qubits;
  tmp.ne = g->n_edges;
  std::vector<double> d(dims, dims + g->n_edges);
  for (double x : d)
    if (!(x >= 1)) return tn_fail(TN_ERR_ARG, "tn_cut_search: dims must be >= 1");
  tn_path_opts o = opts ? *opts : tn_default_opts();
  const double limit = o.max_intermediate > 0 ? (double)o.max_intermediate : (double)(1LL << 24);
  std::vector<int> ord, cut;
  double score = 0;
  int64_t pops = 0;
  int ru = 0;
  PathGraph pg = make_pg(tmp.n, tmp.eu, tmp.ev, d);
  if ((s = path_auto(pg, o, ord, score, pops, ru)) != TN_OK) return s;
  if (o.n_cut_edges > 0) {
    std::vector<double> d2 = d;
    for (int j = 0; j < o.n_cut_edges; ++j) {
      int e = o.cut_edges[j];
      if (e < 0 || e >= tmp.ne) return tn_fail(TN_ERR_ARG, "tn_cut_search: bad cut edge %d", e);
      cut.push_back(e);
      d2[e] = 1;
    }
    PathGraph pg2 = make_pg(tmp.n, tmp.eu, tmp.ev, d2);
    if ((s = path_auto(pg2, o, ord, score, pops, ru)) != TN_OK) return s;
  } else if ((s = choose_cuts(tmp, o, d, o.n_cuts, limit, cut, ord, score, pops, ru)) != TN_OK) {
    return s;
  }
  double slices = 1;
  for (int e : cut) slices *= d[e];
  for (int i = 0; i < tmp.n; ++i) order[i] = ord[i];
  if (cuts)
    for (size_t j = 0; j < cut.size(); ++j) cuts[j] = cut[j];
  *n_cuts = (int32_t)cut.size();
  if (total_cmacs) *total_cmacs = slices * score;
  return TN_OK;
}

extern "C" tn_status tn_cut_search(const tn_graph *g, const double *dims, const tn_path_opts *opts, int32_t *order,
                                     int32_t *cuts, int32_t *n_cuts, double *total_cmacs) {
  return no_throw("tn_cut_search", [&] { return tn_cut_search_impl(g, dims, opts, order, cuts, n_cuts, total_cmacs); });
}

static int64_t dc_of(const tn_circuit *c, int e) { return (int64_t)c->ket.dims[e] * c->bra.dims[e]; }

// ---------------------------------------------------------------------------
// the overlap network: one node per qubit, then boundary nodes merged into neighbours
// ---------------------------------------------------------------------------
static Net identity_net(const tn_circuit *c) {
  Net g;
  g.n = c->n;
  g.ne = c->ne;
  g.eu = c->eu;
  g.ev = c->ev;
  g.legs = c->legs;
  g.eid.resize(c->ne);
  g.dk.resize(c->ne);
  g.db.resize(c->ne);
  for (int e = 0; e < c->ne; ++e) {
    g.eid[e] = e;
    g.dk[e] = c->ket.dims[e];
    g.db[e] = c->bra.dims[e];
  }
  g.rep.resize(c->n);
  g.owner.resize(c->n);
  g.phys.assign(c->n, 2);
  for (int q = 0; q < c->n; ++q) g.rep[q] = g.owner[q] = q;
  g.ket_off = c->ket.node_off;
  g.bra_off = c->bra.node_off;
  g.ket_elems = c->ket.item_elems;
  g.bra_elems = c->bra.item_elems;
  return g;
}

// The double-layer network: qubit q's ket tensor is node q and its bra tensor node n + q, joined
// by an edge of dimension 2 (the physical index sigma_q, id 2 ne + q); ket bond e joins ket nodes
// (id e, dims dk = ket bond, db = 1), its bra bond joins bra nodes (id ne + e, dk = 1, db = bra
// bond). Each node's tensor is the half's node tensor as stored, [sigma, legs in increasing edge
// id], so its legs are [sigma edge, bonds]. These are the sums of Eq. overlap without the
// per-qubit tensors C^q formed first.
static Net double_layer_net(const tn_circuit *c) {
  Net g;
  const int n = c->n, ne = c->ne;
  g.n = 2 * n;
  g.ne = 2 * ne + n;
  g.eu.resize(g.ne);
  g.ev.resize(g.ne);
  g.eid.resize(g.ne);
  g.dk.resize(g.ne);
  g.db.resize(g.ne);
  for (int e = 0; e < ne; ++e) {
    g.eu[e] = c->eu[e];
    g.ev[e] = c->ev[e];
    g.eid[e] = e;
    g.dk[e] = c->ket.dims[e];
    g.db[e] = 1;
    g.eu[ne + e] = n + c->eu[e];
    g.ev[ne + e] = n + c->ev[e];
    g.eid[ne + e] = ne + e;
    g.dk[ne + e] = 1;
    g.db[ne + e] = c->bra.dims[e];
  }
  for (int q = 0; q < n; ++q) {
    const int e = 2 * ne + q;
    g.eu[e] = q;
    g.ev[e] = n + q;
    g.eid[e] = e;
    g.dk[e] = 2;
    g.db[e] = 1;
  }
  g.legs.assign(g.n, {});
  g.rep.resize(g.n);
  g.owner.resize(n);
  g.phys.assign(g.n, 2);              // the unit operand's two values
  g.layer.resize(g.n);
  g.dl_id.resize(g.n);
  for (int v = 0; v < g.n; ++v) g.dl_id[v] = v;
  g.ket_off.resize(g.n);
  g.bra_off.resize(g.n);
  for (int q = 0; q < n; ++q) {
    g.legs[q].push_back(2 * ne + q);
    g.legs[n + q].push_back(2 * ne + q);
    for (int e : c->legs[q]) {
      g.legs[q].push_back(e);
      g.legs[n + q].push_back(ne + e);
    }
    g.rep[q] = g.rep[n + q] = q;
    g.owner[q] = q;
    g.layer[q] = 1;
    g.layer[n + q] = 2;
    g.ket_off[q] = c->ket.node_off[q];
    g.bra_off[q] = 0;                 // unit operand
    g.ket_off[n + q] = 0;             // unit operand
    g.bra_off[n + q] = c->bra.node_off[q];
  }
  g.ket_elems = c->ket.item_elems;
  g.bra_elems = c->bra.item_elems;
  return g;
}

// Renumber the surviving nodes (alive) and edges (eu >= 0) of g compactly, in increasing order;
// nid and eidx map the old ids to the new ones (-1: gone).
static void compact_net(Net &g, const std::vector<char> &alive, std::vector<int> &nid, std::vector<int> &eidx) {
  nid.assign(g.n, -1);
  eidx.assign(g.ne, -1);
  Net h;
  const bool dl = !g.layer.empty();
  for (int v = 0; v < g.n; ++v)
    if (alive[v]) {
      nid[v] = h.n++;
      h.rep.push_back(g.rep[v]);
      h.phys.push_back(g.phys[v]);
      h.ket_off.push_back(g.ket_off[v]);
      h.bra_off.push_back(g.bra_off[v]);
      if (dl) {
        h.layer.push_back(g.layer[v]);
        h.dl_id.push_back(g.dl_id[v]);
      }
    }
  for (int e = 0; e < g.ne; ++e)
    if (g.eu[e] >= 0) {
      eidx[e] = h.ne++;
      h.eu.push_back(nid[g.eu[e]]);
      h.ev.push_back(nid[g.ev[e]]);
      h.eid.push_back(g.eid[e]);
      h.dk.push_back(g.dk[e]);
      h.db.push_back(g.db[e]);
    }
  h.legs.resize(h.n);
  for (int v = 0; v < g.n; ++v)
    if (alive[v])
      for (int e : g.legs[v]) h.legs[nid[v]].push_back(eidx[e]);
  h.owner.resize(g.owner.size());
  for (size_t q = 0; q < g.owner.size(); ++q) h.owner[q] = nid[g.owner[q]];
  h.ket_elems = g.ket_elems;
  h.bra_elems = g.bra_elems;
  h.mk = g.mk;
  h.mb = g.mb;
  g = h;
}

// Merge node v into u through edge a on both halves: U's tensor becomes
// [p_u, p_v, legs_u \ a, legs_v \ a] = sum_a U V, a new slot past the items' current ends.
static void apply_merge(Net &g, int v, int a) {
  const int u = g.eu[a] == v ? g.ev[a] : g.eu[a];
  for (int half = 0; half < 2; ++half) {
    const std::vector<int64_t> &d = half ? g.db : g.dk;
    auto strides = [&](int node, std::vector<int64_t> &st) -> int64_t {
      const auto &L = g.legs[node];
      st.assign(L.size(), 1);
      int64_t x = 1;
      for (int j = (int)L.size() - 1; j >= 0; --j) { st[j] = x; x *= d[L[j]]; }
      return x;
    };
    MergeParams m;
    std::memset(&m, 0, sizeof m);
    std::vector<int64_t> su, sv;
    m.su_p = strides(u, su);
    m.sv_p = strides(v, sv);
    m.pu = g.phys[u];
    m.pv = g.phys[v];
    m.da = (int)d[a];
    m.u_off = half ? g.bra_off[u] : g.ket_off[u];
    m.v_off = half ? g.bra_off[v] : g.ket_off[v];
    int64_t size = (int64_t)m.pu * m.pv;
    for (size_t j = 0; j < g.legs[u].size(); ++j) {
      const int e = g.legs[u][j];
      if (e == a) { m.su_a = su[j]; continue; }
      m.du[m.nu] = (int)d[e];
      m.su[m.nu++] = su[j];
      size *= d[e];
    }
    for (size_t j = 0; j < g.legs[v].size(); ++j) {
      const int e = g.legs[v][j];
      if (e == a) { m.sv_a = sv[j]; continue; }
      m.dv[m.nv] = (int)d[e];
      m.sv[m.nv++] = sv[j];
      size *= d[e];
    }
    m.out_size = size;
    int64_t &ext = half ? g.bra_elems : g.ket_elems;
    m.out_off = ext;
    ext += (size + 1) & ~1LL;
    (half ? g.mb : g.mk).push_back(m);
    (half ? g.bra_off : g.ket_off)[u] = m.out_off;
  }
  std::vector<int> L;
  for (int e : g.legs[u])
    if (e != a) L.push_back(e);
  for (int e : g.legs[v]) {
    if (e == a) continue;
    L.push_back(e);
    (g.eu[e] == v ? g.eu[e] : g.ev[e]) = u;
  }
  g.legs[u] = L;
  g.legs[v].clear();
  g.phys[u] *= g.phys[v];
  g.eu[a] = g.ev[a] = -1;
  for (int &o : g.owner)
    if (o == v) o = u;
}

// Repeatedly merge a not-yet-merged node v of degree <= 2 into the neighbour u across its widest
// edge a when v's other legs are no wider than a (the merged tensor is no larger than u's), the
// physical dimension stays <= 8, no parallel edge appears, no kept edge (an explicit cut) is
// merged away, and at least two nodes remain. Then renumber nodes and edges compactly.
static void merge_nodes(Net &g, const std::vector<char> &keep_edge) {
  std::vector<char> alive(g.n, 1);
  int n_alive = g.n;
  auto other = [&](int e, int x) { return g.eu[e] == x ? g.ev[e] : g.eu[e]; };
  for (bool did = true; did && n_alive > 2;) {
    did = false;
    for (int v = 0; v < g.n && !did; ++v) {
      if (!alive[v] || g.phys[v] != 2 || g.legs[v].empty() || g.legs[v].size() > 2) continue;
      int best = -1;
      for (int a : g.legs[v]) {
        if (keep_edge[g.eid[a]]) continue;
        const int u = other(a, v);
        if (g.phys[u] * g.phys[v] > 8) continue;
        if (g.legs[u].size() + g.legs[v].size() - 2 > TN_MAXMLEGS) continue;
        int64_t rest = 1;
        bool parallel = false;
        for (int e : g.legs[v]) {
          if (e == a) continue;
          rest *= g.dc(e);
          const int x = other(e, v);
          if (x == u) parallel = true;
          for (int f : g.legs[u])
            if (other(f, u) == x) parallel = true;
        }
        if (parallel || rest > g.dc(a)) continue;
        if (best < 0 || g.dc(a) > g.dc(best)) best = a;
      }
      if (best < 0) continue;
      apply_merge(g, v, best);
      alive[v] = 0;
      --n_alive;
      did = true;
    }
  }
  std::vector<int> nid, eidx;
  compact_net(g, alive, nid, eidx);
}

// Join two same-layer nodes of a double-layer network, v into u through their edge a, in that
// layer's half: u's tensor becomes [legs_u \ a, legs_v \ a] = sum_a U V, computed exactly in FP64
// (once per batch for ket tensors, for every bitstring for bra tensors) in a new slot past the
// half's item.
static void apply_layer_merge(Net &g, int u, int v, int a) {
  const int half = g.layer[u] == 2 ? 1 : 0;
  auto strides = [&](int node, std::vector<int64_t> &st) -> int64_t {
    const auto &L = g.legs[node];
    st.assign(L.size(), 1);
    int64_t x = 1;
    for (int j = (int)L.size() - 1; j >= 0; --j) { st[j] = x; x *= g.dc(L[j]); }
    return x;
  };
  MergeParams m;
  std::memset(&m, 0, sizeof m);
  std::vector<int64_t> su, sv;
  m.su_p = strides(u, su);
  m.sv_p = strides(v, sv);
  m.pu = m.pv = 1;
  m.da = (int)g.dc(a);
  m.u_off = half ? g.bra_off[u] : g.ket_off[u];
  m.v_off = half ? g.bra_off[v] : g.ket_off[v];
  int64_t size = 1;
  for (size_t j = 0; j < g.legs[u].size(); ++j) {
    const int e = g.legs[u][j];
    if (e == a) { m.su_a = su[j]; continue; }
    m.du[m.nu] = (int)g.dc(e);
    m.su[m.nu++] = su[j];
    size *= g.dc(e);
  }
  for (size_t j = 0; j < g.legs[v].size(); ++j) {
    const int e = g.legs[v][j];
    if (e == a) { m.sv_a = sv[j]; continue; }
    m.dv[m.nv] = (int)g.dc(e);
    m.sv[m.nv++] = sv[j];
    size *= g.dc(e);
  }
  m.out_size = size;
  int64_t &ext = half ? g.bra_elems : g.ket_elems;
  m.out_off = ext;
  ext += (size + 1) & ~1LL;
  (half ? g.mb : g.mk).push_back(m);
  (half ? g.bra_off : g.ket_off)[u] = m.out_off;
  std::vector<int> L;
  for (int e : g.legs[u])
    if (e != a) L.push_back(e);
  for (int e : g.legs[v]) {
    if (e == a) continue;
    L.push_back(e);
    (g.eu[e] == v ? g.eu[e] : g.ev[e]) = u;
  }
  g.legs[u] = L;
  g.legs[v].clear();
  g.eu[a] = g.ev[a] = -1;
  for (int &o : g.owner)
    if (o == v) o = u;
}

// Joining partial paths (supplement, the discussion of Assumption 3: partial paths that grow
// separately and are joined by one pairwise contraction), as a pass over the path Algorithm 1 found
// on a double-layer network. Where the path absorbs two nodes u, v of the same layer in a row and
// they share one edge a that is not cut, the pair can be contracted on its own first (a second
// partial path {u, v}) and joined to the main path in one step. The pass does so when that lowers
// both the complex multiply-adds (the pair's own contraction counted once per bitstring for bra
// tensors) and the elements the steps read and write, then tries the joined node with the next one.
// The amplitude is the same sum in another grouping; the largest intermediate does not grow (the
// joined step reads step j's input and writes step j + 1's output).
static void join_paths(tn_plan *p) {
  Net &g = p->net;
  std::vector<char> is_cut(g.ne, 0), open(g.ne, 0), alive(g.n, 1);
  for (int e : p->cuts) is_cut[e] = 1;
  std::vector<int> ord = p->order;
  auto other = [&](int e, int x) { return g.eu[e] == x ? g.ev[e] : g.eu[e]; };
  // K (legs of L open now) and N (legs of L not open and not cut), as products of dims
  auto split = [&](const std::vector<int> &L, int skip, double &K, double &N) {
    K = N = 1;
    for (int e : L) {
      if (e == skip || is_cut[e]) continue;
      if (open[e]) K *= (double)g.dc(e);
      else N *= (double)g.dc(e);
    }
  };
  double oprod = 1;   // elements of the current intermediate
  size_t j = 0;
  while (j + 1 < ord.size()) {
    const int u = ord[j], v = ord[j + 1];
    int a = -1, shared = 0;
    for (int e : g.legs[u])
      if (other(e, u) == v) { a = e; ++shared; }
    bool joined = false;
    if (g.layer[u] == g.layer[v] && shared == 1 && !is_cut[a] && (int)g.legs[u].size() - 1 <= TN_MERGE_MAXLEGS &&
        (int)g.legs[v].size() - 1 <= TN_MERGE_MAXLEGS) {
      double K1, N1, K2, N2, Kw, Nw, Kv, Nv;
      split(g.legs[u], -1, K1, N1);
      const double M1 = oprod / K1;
      // the intermediate after u: u's open legs closed, its new ones (a among them) opened
      split(g.legs[v], a, Kv, Nv);
      K2 = Kv * (double)g.dc(a);   // v's legs open after u: a, and those already open before u
      N2 = Nv;
      const double M2 = M1 * N1 / K2;
      Kw = K1 * Kv;
      Nw = (N1 / (double)g.dc(a)) * Nv;
      const double Mw = oprod / Kw;
      const bool first = j == 0;
      const double seq_mac = (first ? 0 : M1 * K1 * N1) + M2 * K2 * N2;
      const double seq_el = (first ? 0 : M1 * K1 + M1 * N1) + M2 * K2 + M2 * N2;
      double pair = 1;   // the pair's own contraction: prod of the dims of all legs of u and v, a once
      for (int e : g.legs[u]) pair *= (double)g.dc(e);
      for (int e : g.legs[v])
        if (e != a) pair *= (double)g.dc(e);
      const double w_mac = (first ? 0 : Mw * Kw * Nw) + (g.layer[u] == 2 ? pair : 0);
      const double w_el = first ? 0 : Mw * Kw + Mw * Nw;
      if (w_mac <= seq_mac && w_el <= seq_el && (w_mac < seq_mac || w_el < seq_el)) {
        apply_layer_merge(g, u, v, a);
        alive[v] = 0;
        ord.erase(ord.begin() + (long)j + 1);
        joined = true;
      }
    }
    if (joined) continue;
    double K1, N1;
    split(g.legs[u], -1, K1, N1);
    oprod = oprod / K1 * N1;
    for (int e : g.legs[u])
      if (!is_cut[e]) open[e] = !open[e];
    ++j;
  }
  std::vector<int> nid, eidx;
  compact_net(g, alive, nid, eidx);
  for (int &x : ord) x = nid[x];
  for (int &e : p->cuts) e = eidx[e];
  p->order = ord;
}

static tn_status tn_merge_search_impl(const tn_graph *g, const int32_t *ket_dims, const int32_t *bra_dims,
                                     const tn_path_opts *opts, int32_t *owner, int32_t *n_nodes, int32_t *order,
                                     int32_t *n_cuts, double *total_cmacs) {
  if (!g || !ket_dims || !bra_dims || !owner || !n_nodes || !order)
    return tn_fail(TN_ERR_ARG, "tn_merge_search: NULL argument");
  Net net;
  tn_status s = check_graph(g, net.eu, net.ev, net.legs);
  if (s != TN_OK) return s;
  net.n = g->n_qubits;
  net.ne = g->n_edges;
  net.eid.resize(net.ne);
  net.dk.resize(net.ne);
  net.db.resize(net.ne);
  for (int e = 0; e < net.ne; ++e) {
    if (ket_dims[e] < 1 || bra_dims[e] < 1) return tn_fail(TN_ERR_ARG, "tn_merge_search: dims must be >= 1");
    net.eid[e] = e;
    net.dk[e] = ket_dims[e];
    net.db[e] = bra_dims[e];
  }
  net.rep.resize(net.n);
  net.owner.resize(net.n);
  net.phys.assign(net.n, 2);
  net.ket_off.assign(net.n, 0);
  net.bra_off.assign(net.n, 0);
  for (int q = 0; q < net.n; ++q) net.rep[q] = net.owner[q] = q;
  tn_path_opts o = opts ? *opts : tn_default_opts();
  std::vector<char> keep(net.ne, 0);
  for (int j = 0; j < o.n_cut_edges; ++j) {
    const int e = o.cut_edges ? o.cut_edges[j] : -1;
    if (e < 0 || e >= net.ne) return tn_fail(TN_ERR_ARG, "tn_merge_search: bad cut edge %d", e);
    keep[e] = 1;
  }
  if (!o.no_merge) merge_nodes(net, keep);
  std::vector<double> d(net.ne);
  for (int e = 0; e < net.ne; ++e) d[e] = (double)net.dc(e);
  const double limit = o.max_intermediate > 0 ? (double)o.max_intermediate : (double)(1LL << 24);
  std::vector<int> ord, cut;
  double score = 0;
  int64_t pops = 0;
  int ru = 0;
  PathGraph pg = make_pg(net.n, net.eu, net.ev, d);
  if ((s = path_auto(pg, o, ord, score, pops, ru)) != TN_OK) return s;
  if (o.n_cut_edges > 0) {
    for (int e = 0; e < net.ne; ++e)
      if (keep[net.eid[e]]) { cut.push_back(e); d[e] = 1; }
    PathGraph pg2 = make_pg(net.n, net.eu, net.ev, d);
    if ((s = path_auto(pg2, o, ord, score, pops, ru)) != TN_OK) return s;
  } else if ((s = choose_cuts(net, o, d, o.n_cuts, limit, cut, ord, score, pops, ru)) != TN_OK) {
    return s;
  }
  double slices = 1;
  for (int e : cut) slices *= (double)net.dc(e);
  for (int q = 0; q < g->n_qubits; ++q) owner[q] = net.rep[net.owner[q]];
  *n_nodes = net.n;
  for (int j = 0; j < net.n; ++j) order[j] = net.rep[ord[j]];
  if (n_cuts) *n_cuts = (int32_t)cut.size();
  if (total_cmacs) *total_cmacs = slices * score;
  return TN_OK;
}

extern "C" tn_status tn_merge_search(const tn_graph *g, const int32_t *ket_dims, const int32_t *bra_dims,
                                       const tn_path_opts *opts, int32_t *owner, int32_t *n_nodes, int32_t *order,
                                       int32_t *n_cuts, double *total_cmacs) {
  return no_throw("tn_merge_search", [&] { return tn_merge_search_impl(g, ket_dims, bra_dims, opts, owner, n_nodes, order, n_cuts, total_cmacs); });
}

// Every device index a compiled plan can produce, checked on the host before any launch: node
// tensors inside their items, the tables' offsets inside their node's tensor, each step's input
// and output inside the intermediate's item stride, the merges' reads and writes inside their
// slots. A violation is an internal error of the compiler, reported instead of launched.
static tn_status validate_plan(const tn_plan *p) {
  const Net &g = p->net;
  const std::vector<int32_t> &tab = p->tab_host;
  auto bad = [](const char *what, int j, long long v, long long lim) {
    return tn_fail(TN_ERR_UNSUPPORTED, "plan check failed: %s (step or node %d: %lld >= %lld)", what, j, v, lim);
  };
  auto tmax = [&](int64_t off, int64_t n) {
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) m = std::max<int64_t>(m, tab[off + i]);
    return m;
  };
  const auto layer_of = [&](int i) { return g.layer.empty() ? 0 : g.layer[i]; };
  // a double-layer node's own tensor (its legs' dims dc) in its half's item; the unit operand
  // (two values) in the other slot
  auto own_size = [&](int i) {
    int64_t t = 1;
    for (int e : g.legs[i]) t *= g.dc(e);
    return t;
  };
  for (int i = 0; i < g.n; ++i) {
    int64_t sk = g.phys[i], sb = g.phys[i];
    if (layer_of(i) == 1) { sk = own_size(i); sb = 2; }
    else if (layer_of(i) == 2) { sk = 2; sb = own_size(i); }
    else for (int e : g.legs[i]) { sk *= g.dk[e]; sb *= g.db[e]; }
    const int64_t klim = layer_of(i) == 2 ? 2 : g.ket_elems, blim = layer_of(i) == 1 ? 2 : g.bra_elems;
    if (g.ket_off[i] + sk > klim) return bad("ket node tensor outside the item", i, g.ket_off[i] + sk, klim);
    if (g.bra_off[i] + sb > blim) return bad("bra node tensor outside the item", i, g.bra_off[i] + sb, blim);
  }
  for (int h = 0; h < 2; ++h) {
    const std::vector<MergeParams> &ms = h ? g.mb : g.mk;
    const int64_t lim = h ? g.bra_elems : g.ket_elems;
    for (size_t t = 0; t < ms.size(); ++t) {
      const MergeParams &m = ms[t];
      int64_t ru = (int64_t)(m.pu - 1) * m.su_p + (int64_t)(m.da - 1) * m.su_a, rv = (int64_t)(m.pv - 1) * m.sv_p + (int64_t)(m.da - 1) * m.sv_a;
      for (int q = 0; q < m.nu; ++q) ru += (int64_t)(m.du[q] - 1) * m.su[q];
      for (int q = 0; q < m.nv; ++q) rv += (int64_t)(m.dv[q] - 1) * m.sv[q];
      if (ru >= (int64_t)m.pu * m.su_p) return bad("merge reads outside U", (int)t, ru, (int64_t)m.pu * m.su_p);
      if (rv >= (int64_t)m.pv * m.sv_p) return bad("merge reads outside V", (int)t, rv, (int64_t)m.pv * m.sv_p);
      if (m.u_off + m.pu * m.su_p > lim || m.v_off + m.pv * m.sv_p > lim || m.out_off + m.out_size > lim)
        return bad("merge slot outside the item", (int)t, m.out_off + m.out_size, lim);
    }
  }
  for (size_t j = 0; j < p->steps.size(); ++j) {
    const StepParams &s = p->steps[j];
    const int i = p->order[j];
    int64_t tk = s.phys * s.ket_sig, tb = s.phys * s.bra_sig;   // the node's tensor sizes
    if (layer_of(i) == 1) { tk = own_size(i); tb = 2; }
    else if (layer_of(i) == 2) { tk = 2; tb = own_size(i); }
    const int64_t ka = tmax(s.t_sa, p->n_slices) + tmax(s.t_bna, s.N) + (j ? tmax(s.t_bka, s.K) : 0) +
                       (s.phys - 1) * s.ket_sig;
    const int64_t kb = tmax(s.t_sb, p->n_slices) + tmax(s.t_bnb, s.N) + (j ? tmax(s.t_bkb, s.K) : 0) +
                       (s.phys - 1) * s.bra_sig;
    if (ka >= tk) return bad("ket offsets outside the node tensor", (int)j, ka, tk);
    if (kb >= tb) return bad("bra offsets outside the node tensor", (int)j, kb, tb);
    if (s.ket_off != g.ket_off[i] || s.bra_off != g.bra_off[i]) return bad("node offset mismatch", (int)j, 0, 0);
    if (j > 0 && s.M * s.K > p->maxT) return bad("step input larger than the item stride", (int)j, s.M * s.K, p->maxT);
    int64_t orow = 0;
    for (int r = 0; r < s.n_rest; ++r) orow += (int64_t)(s.rest_dim[r] - 1) * s.rest_ostride[r];
    const int64_t omax = orow + tmax(s.t_ocol, s.N);
    if (omax >= p->maxT) return bad("step output outside the item stride", (int)j, omax, p->maxT);
    if (s.box_tm > 0) {
      // box tiles: box_tm divides M along the digits (trailing digits whole, then one divisor),
      // and the sorted write table holds every (r, n) of a tile once
      int64_t q = s.box_tm;
      for (int r = s.n_rest - 1; r >= 0 && q > 1; --r) {
        const int64_t d = s.rest_dim[r];
        if (q % d == 0) { q /= d; continue; }
        if (d % q != 0) return bad("box tile not aligned to the rest digits", (int)j, s.box_tm, s.M);
        q = 1;
      }
      if (q != 1 || s.M % s.box_tm != 0 || s.box_tm >= (1 << 14) || s.t_wperm % 2 != 0)
        return bad("box tile does not divide the rows", (int)j, s.box_tm, s.M);
      std::vector<char> seen((size_t)s.box_tm * s.N, 0);
      const int64_t tot = (int64_t)s.box_tm * s.N;
      for (int64_t e = 0; e < tot; ++e) {
        const uint32_t pr = (uint32_t)tab[s.t_wperm + 2 * e];
        const int64_t r = (pr >> 16) & 0x3fffu, nn = pr & 0xffffu;
        if (r >= s.box_tm || nn >= s.N || seen[r * s.N + nn]) return bad("box write table", (int)j, e, tot);
        seen[r * s.N + nn] = 1;
        int64_t orl = 0, x = r;
        for (int q = s.n_rest - 1; q >= 0; --q) { orl += (x % s.rest_dim[q]) * s.rest_ostride[q]; x /= s.rest_dim[q]; }
        if (tab[s.t_wperm + 2 * e + 1] != orl + tab[s.t_ocol + nn]) return bad("box write offset", (int)j, e, tot);
        if ((pr >> 30) & 1u) {   // a pair: the next entry is (r, n + 1) at the next offset, both even
          const uint32_t p1 = (uint32_t)tab[s.t_wperm + 2 * e + 2];
          if (e % 2 || e + 1 >= tot || ((p1 >> 16) & 0x3fffu) != r || (p1 & 0xffffu) != nn + 1 || nn % 2 ||
              tab[s.t_wperm + 2 * e + 3] != tab[s.t_wperm + 2 * e + 1] + 1 || tab[s.t_wperm + 2 * e + 1] % 2)
            return bad("box write pair", (int)j, e, tot);
        }
      }
    }
  }
  return TN_OK;
}

static tn_status compile_plan(tn_plan *p) {
  const Net &c = p->net;
  const int n = c.n;
  std::vector<int> pos(n);
  for (int j = 0; j < n; ++j) pos[p->order[j]] = j;
  std::vector<char> is_cut(c.ne, 0);
  for (int e : p->cuts) is_cut[e] = 1;
  std::vector<int64_t> cut_stride(p->cuts.size());
  {
    double sd = 1;   // checked in floating point first: the product can overflow int64
    for (int e : p->cuts) sd *= (double)c.dc(e);
    // every step holds two int32 offset tables over the slices
    if (sd * 2.0 * n >= (double)(1LL << 31))
      return tn_fail(TN_ERR_UNSUPPORTED,
                     "%.3g slices: their offset tables exceed the plan's table limit; allow larger intermediates "
                     "(max_intermediate) or cap the bonds (chi)", sd);
    int64_t s = 1;
    for (int j = (int)p->cuts.size() - 1; j >= 0; --j) { cut_stride[j] = s; s *= c.dc(p->cuts[j]); }
    p->n_slices = s;
  }
  auto &tab = p->tab_host;
  tab.clear();
  auto push_tab = [&](const std::vector<int64_t> &v) -> int64_t {
    int64_t off = (int64_t)tab.size();
    for (int64_t x : v) tab.push_back((int32_t)x);
    return off;
  };
  // per-node ket/bra strides of each leg
  auto leg_strides = [&](int i, const std::vector<int64_t> &dims, std::vector<int64_t> &st) -> int64_t {
    const auto &L = c.legs[i];
    st.assign(L.size(), 1);
    int64_t s = 1;
    for (int j = (int)L.size() - 1; j >= 0; --j) { st[j] = s; s *= dims[L[j]]; }
    return s;
  };
  // double-layer nodes: one tensor with leg dims dc in the node's own slot (1 ket, 2 bra)
  const auto layer_of = [&](int i) { return c.layer.empty() ? 0 : c.layer[i]; };
  std::vector<int64_t> dcv(c.ne);
  for (int e = 0; e < c.ne; ++e) dcv[e] = c.dc(e);
  // tables over a list of legs of node i: offsets into ket / bra for each multi-index
  auto leg_tables = [&](int i, const std::vector<int> &legs, std::vector<int64_t> &ta, std::vector<int64_t> &tb) {
    if (layer_of(i) != 0) {
      std::vector<int64_t> sd;
      leg_strides(i, dcv, sd);
      int64_t total = 1;
      for (int e : legs) total *= c.dc(e);
      ta.assign(total, 0);
      tb.assign(total, 0);
      std::vector<int64_t> &own = layer_of(i) == 1 ? ta : tb;
      for (int64_t idx = 0; idx < total; ++idx) {
        int64_t r = idx, o = 0;
        for (int j = (int)legs.size() - 1; j >= 0; --j) {
          const int e = legs[j];
          const int64_t d = c.dc(e);
          const int li = (int)(std::find(c.legs[i].begin(), c.legs[i].end(), e) - c.legs[i].begin());
          o += (r % d) * sd[li];
          r /= d;
        }
        own[idx] = o;
      }
      return;
    }
    std::vector<int64_t> sk, sb;
    leg_strides(i, c.dk, sk);
    leg_strides(i, c.db, sb);
    int64_t total = 1;
    for (int e : legs) total *= c.dc(e);
    ta.assign(total, 0);
    tb.assign(total, 0);
    for (int64_t idx = 0; idx < total; ++idx) {
      int64_t r = idx, oa = 0, ob = 0;
      for (int j = (int)legs.size() - 1; j >= 0; --j) {
        int e = legs[j];
        int64_t d = c.dc(e), cval = r % d;
        r /= d;
        int li = (int)(std::find(c.legs[i].begin(), c.legs[i].end(), e) - c.legs[i].begin());
        int64_t db = c.db[e];
        oa += (cval / db) * sk[li];
        ob += (cval % db) * sb[li];
      }
      ta[idx] = oa;
      tb[idx] = ob;
    }
  };
  auto slice_tables = [&](int i, std::vector<int64_t> &sa, std::vector<int64_t> &sbv) {
    std::vector<int64_t> sk, sb;
    leg_strides(i, c.dk, sk);
    leg_strides(i, c.db, sb);
    sa.assign(p->n_slices, 0);
    sbv.assign(p->n_slices, 0);
    if (layer_of(i) != 0) {
      std::vector<int64_t> sd;
      leg_strides(i, dcv, sd);
      std::vector<int64_t> &own = layer_of(i) == 1 ? sa : sbv;
      for (int64_t s = 0; s < p->n_slices; ++s)
        for (size_t j = 0; j < p->cuts.size(); ++j) {
          const int e = p->cuts[j];
          auto it = std::find(c.legs[i].begin(), c.legs[i].end(), e);
          if (it == c.legs[i].end()) continue;
          own[s] += ((s / cut_stride[j]) % c.dc(e)) * sd[(int)(it - c.legs[i].begin())];
        }
      return;
    }
    for (int64_t s = 0; s < p->n_slices; ++s) {
      for (size_t j = 0; j < p->cuts.size(); ++j) {
        int e = p->cuts[j];
        auto it = std::find(c.legs[i].begin(), c.legs[i].end(), e);
        if (it == c.legs[i].end()) continue;
        int li = (int)(it - c.legs[i].begin());
        int64_t cval = (s / cut_stride[j]) % c.dc(e);
        int64_t db = c.db[e];
        sa[s] += (cval / db) * sk[li];
        sbv[s] += (cval % db) * sb[li];
      }
    }
  };
  auto new_legs_of = [&](int i, const std::vector<char> &open) {
    std::vector<int> nl;
    for (int e : c.legs[i])
      if (!is_cut[e] && !open[e]) nl.push_back(e);
    // later-absorbed neighbours first, so the next consumer's legs are innermost
    std::sort(nl.begin(), nl.end(), [&](int a, int b) {
      int oa = c.eu[a] == i ? c.ev[a] : c.eu[a];
      int ob = c.eu[b] == i ? c.ev[b] : c.eu[b];
      return pos[oa] > pos[ob];
    });
    return nl;
  };
  p->steps.clear();
  p->step_mkn.clear();
  p->step_layer.clear();
  // pass 1: per step the rest, shared and new legs; the input layout of step j is
  // [rest_j, shared_j], both in the order the legs were created
  std::vector<std::vector<int>> R(n), Sh(n), Nw(n);
  {
    std::vector<char> open(c.ne, 0);
    std::vector<int> cur;
    for (int j = 0; j < n; ++j) {
      const int i = p->order[j];
      for (int e : cur) ((c.eu[e] == i || c.ev[e] == i) ? Sh[j] : R[j]).push_back(e);
      Nw[j] = new_legs_of(i, open);
      for (int e : Sh[j]) open[e] = 0;
      for (int e : Nw[j]) open[e] = 1;
      cur = R[j];
      cur.insert(cur.end(), Nw[j].begin(), Nw[j].end());
    }
  }
  auto prod_dims = [&](const std::vector<int> &legs) {
    int64_t x = 1;
    for (int e : legs) x *= c.dc(e);
    return x;
  };
  // pass 2: kernels' parameters; output strides are those of the next step's input layout
  double cmacs = 0, bytes = 0;
  int64_t maxT = 1;
  for (int j = 0; j < n; ++j) {
    const int i = p->order[j];
    StepParams s;
    std::memset(&s, 0, sizeof s);
    const int64_t M = prod_dims(R[j]), K = prod_dims(Sh[j]), N = prod_dims(Nw[j]);
    s.M = M; s.K = K; s.N = N;
    if ((int)R[j].size() > TN_MAXREST) return tn_fail(TN_ERR_UNSUPPORTED, "step %d has %zu rest legs", j, R[j].size());
    std::vector<int> Lnext;   // input layout of step j+1 (empty after the last step)
    if (j + 1 < n) {
      Lnext = R[j + 1];
      Lnext.insert(Lnext.end(), Sh[j + 1].begin(), Sh[j + 1].end());
    }
    auto ostride = [&](int e) -> int64_t {
      int64_t st = 1;
      for (int q = (int)Lnext.size() - 1; q >= 0; --q) {
        if (Lnext[q] == e) return st;
        st *= c.dc(Lnext[q]);
      }
      return 0;
    };
    s.n_rest = (int)R[j].size();
    s.rest_pow2 = 1;
    for (size_t r = 0; r < R[j].size(); ++r) {
      const int64_t d = c.dc(R[j][r]);
      s.rest_dim[r] = (int)d;
      s.rest_ostride[r] = (int)ostride(R[j][r]);
      int lg = 0;
      while ((1LL << lg) < d) ++lg;
      s.rest_log2[r] = lg;
      if ((1LL << lg) != d) s.rest_pow2 = 0;
    }
    std::vector<int64_t> ocol(N, 0);
    for (int64_t nn = 0; nn < N; ++nn) {
      int64_t r = nn, off = 0;
      for (int q = (int)Nw[j].size() - 1; q >= 0; --q) {
        const int64_t d = c.dc(Nw[j][q]);
        off += (r % d) * ostride(Nw[j][q]);
        r /= d;
      }
      ocol[nn] = off;
    }
    std::vector<int64_t> ka, kb, na, nb, sa, sb;
    leg_tables(i, Sh[j], ka, kb);
    leg_tables(i, Nw[j], na, nb);
    slice_tables(i, sa, sb);
    s.t_ocol = push_tab(ocol);
    s.t_bka = push_tab(ka);
    s.t_bkb = push_tab(kb);
    s.t_bna = push_tab(na);
    s.t_bnb = push_tab(nb);
    s.t_sa = push_tab(sa);
    s.t_sb = push_tab(sb);
    if (j > 0 && K * N <= TN_BOX_MAXKN && N <= TN_BOX_MAXN) {
      // Row tiles of the box-tiled streaming kernel: the trailing rest digits (fastest first),
      // the last one taken in part (a divisor of its dim), so that m = t * tm + r splits the
      // digits of m and orow(m) = orow(t * tm) + orow(r); at most TN_BOX_ROWS_ELEMS / (2 K + N) rows.
      const int64_t lim = std::max<int64_t>(1, TN_BOX_ROWS_ELEMS / (2 * K + N));
      int64_t tm = 1;
      for (int r = s.n_rest - 1; r >= 0; --r) {
        const int64_t d = s.rest_dim[r];
        if (tm * d <= lim) { tm *= d; continue; }
        int64_t f = lim / tm;
        while (f > 1 && d % f != 0) --f;
        tm *= f;
        break;
      }
      // the tile's outputs in increasing output offset (ties in row-major order)
      std::vector<int64_t> orl(tm);
      for (int64_t r = 0; r < tm; ++r) {
        int64_t x = r, off = 0;
        for (int q = s.n_rest - 1; q >= 0; --q) { off += (x % s.rest_dim[q]) * s.rest_ostride[q]; x /= s.rest_dim[q]; }
        orl[r] = off;
      }
      std::vector<int64_t> perm(tm * N);
      for (int64_t e = 0; e < tm * N; ++e) perm[e] = e;
      std::stable_sort(perm.begin(), perm.end(), [&](int64_t x, int64_t y) {
        return orl[x / N] + ocol[x % N] < orl[y / N] + ocol[y % N];
      });
      // per output, in that order: (r << 16 | n) and its offset orow(r) + ocol(n) in the tile; bit 30
      // of an even entry marks it and the next as one pair (same row, columns n and n + 1 with n
      // even, offsets d and d + 1 with d even), which the kernel moves as one 16-byte value
      std::vector<int64_t> tabw(2 * tm * N);
      for (int64_t e = 0; e < tm * N; ++e) {
        const int64_t r = perm[e] / N, nn = perm[e] % N;
        tabw[2 * e] = (r << 16) | nn;
        tabw[2 * e + 1] = orl[r] + ocol[nn];
      }
      for (int64_t e = 0; e + 1 < tm * N; e += 2) {
        const int64_t r0 = perm[e] / N, n0 = perm[e] % N, r1 = perm[e + 1] / N, n1 = perm[e + 1] % N;
        if (r1 == r0 && n1 == n0 + 1 && n0 % 2 == 0 && tabw[2 * e + 3] == tabw[2 * e + 1] + 1 && tabw[2 * e + 1] % 2 == 0)
          tabw[2 * e] |= (int64_t)1 << 30;
      }
      s.box_tm = (int)tm;
      if (tab.size() & 1) tab.push_back(0);   // 8-byte aligned: the kernel reads the entries in pairs
      s.t_wperm = push_tab(tabw);
    }
    std::vector<int64_t> skk, sbb;
    s.ket_sig = leg_strides(i, c.dk, skk);
    s.bra_sig = leg_strides(i, c.db, sbb);
    s.phys = c.phys[i];
    if (layer_of(i) != 0) {
      // sum over the unit operand's two values: own[x] * 1 + own[x] * 0 (own stride 0, unit stride 1)
      s.phys = 2;
      s.ket_sig = layer_of(i) == 1 ? 0 : 1;
      s.bra_sig = layer_of(i) == 1 ? 1 : 0;
    }
    s.ket_off = c.ket_off[i];
    s.bra_off = c.bra_off[i];
    p->steps.push_back(s);
    p->step_layer.push_back(layer_of(i));
    p->step_mkn.push_back({M, K, N});
    if (j > 0) {
      cmacs += (double)M * K * N;
      bytes += 8.0 * ((double)M * K + (double)M * N);
      p->maxKN = std::max(p->maxKN, K * N);
    }
    maxT = std::max(maxT, M * N);
  }
  maxT = (maxT + 7) & ~7LL;             // item strides stay 16-byte aligned in every format
  p->maxKN = (p->maxKN + 1) & ~1LL;
  if (maxT >= (1LL << 31) || (int64_t)tab.size() >= (1LL << 31))
    return tn_fail(TN_ERR_UNSUPPORTED, "intermediate of %lld elements exceeds the 2^31 index range; add cuts",
                   (long long)maxT);
  p->maxT = maxT;
  p->cmacs = cmacs * (double)p->n_slices;
  p->bytes = bytes * (double)p->n_slices;
  return validate_plan(p);
}

static void fill_info(const tn_plan *p, tn_plan_info *info) {
  if (!info) return;
  std::memset(info, 0, sizeof *info);
  info->n_qubits = p->c->n;
  info->n_steps = p->net.n - 1;
  info->n_nodes = p->net.n;
  info->n_cuts = (int32_t)p->cuts.size();
  info->n_slices = p->n_slices;
  info->score = p->score;
  info->cmacs = p->cmacs;
  info->flops = 8.0 * p->cmacs;
  info->bytes_c64 = p->bytes;
  info->max_intermediate = p->maxT;
  info->states_expanded = p->pops;
  info->max_rank_used = p->rank_used;
  info->chunk_bitstrings = p->chunk[0];
  info->workspace_bytes = p->ws_bytes[0];
}

// workspace of `chunk` bitstrings with `slices` slices each per launch group
int64_t plan_ws_bytes(const tn_plan *p, int kind, int64_t chunk, int64_t slices) {
  const tn_circuit *c = p->c;
  const int64_t el = kind == 0 ? 16 : 8;
  const int words = (c->n + 63) / 64;
  int64_t b = 0;
  b += chunk * words * 8;                                   // bits
  b += chunk * p->net.bra_elems * 16;                       // bra FP64 (with merged nodes)
  if (kind) b += chunk * p->net.bra_elems * 8;              // bra c64 copy
  if (p->net.merged()) b += p->net.ket_elems * (kind ? 24 : 16);   // the ket with merged nodes
  b += chunk * std::max<int64_t>(c->bra.max_work, 1) * 16;  // SVD work beyond shared memory
  // ping-pong intermediates (complex64 or three bf16 pieces per real on the complex64 paths)
  b += 2 * chunk * slices * p->maxT * (kind ? 12 : el);
  if (kind) b += chunk * slices * p->maxKN * 24;            // overlap tensors of the tensor-core steps
  b += chunk * 16 + 4096;                                   // results, flags
  return b;
}

// The host part of a plan of circuit c (its programs built): network, path, cuts, compiled and
// checked steps, batch sizes. No device work; on failure p is left for the caller to delete.
static tn_status plan_host(tn_circuit *c, const tn_path_opts &o, tn_plan *p) {
  const double limit = o.max_intermediate > 0 ? (double)o.max_intermediate : (double)(1LL << 24);
  if (o.n_cut_edges > 0 && !o.cut_edges) return tn_fail(TN_ERR_ARG, "tn_path: cut_edges is NULL");
  if (o.layers < 0 || o.layers > 2) return tn_fail(TN_ERR_ARG, "tn_path: layers must be 1 or 2");
  const bool two_layers = o.layers == 2;
  if (two_layers && o.n_cut_edges > 0)
    return tn_fail(TN_ERR_UNSUPPORTED, "tn_path: explicit cut edges are not accepted with the double-layer network");
  std::vector<char> keep(c->ne, 0);   // explicit cut edges stay edges of the network
  for (int j = 0; j < o.n_cut_edges; ++j) {
    const int e = o.cut_edges[j];
    if (e < 0 || e >= c->ne || keep[e]) return tn_fail(TN_ERR_ARG, "tn_path: bad or repeated cut edge %d", e);
    keep[e] = 1;
  }
  if (two_layers && 2 * c->n > 256)
    return tn_fail(TN_ERR_UNSUPPORTED, "tn_path: the double-layer network of %d qubits has more than 256 nodes", c->n);
  p->c = c;
  p->generation = c->generation;
  if (two_layers) {
    p->net = double_layer_net(c);
  } else {
    p->net = identity_net(c);
    if (!o.no_merge) merge_nodes(p->net, keep);
  }
  const Net &g = p->net;
  std::vector<double> dims(g.ne);
  for (int e = 0; e < g.ne; ++e) dims[e] = (double)g.dc(e);
  PathGraph pg = make_pg(g.n, g.eu, g.ev, dims);
  int64_t pops = 0;
  tn_status s = path_auto(pg, o, p->order, p->score, pops, p->rank_used);
  p->pops = pops;
  if (s != TN_OK) return s;
  // cuts: explicit, counted or automatic (thinnest frontier first), then the path of the cut network
  if (o.n_cut_edges > 0) {
    for (int j = 0; j < o.n_cut_edges; ++j)
      for (int e = 0; e < g.ne; ++e)
        if (g.eid[e] == o.cut_edges[j]) p->cuts.push_back(e);
    std::vector<double> cd2 = dims;
    for (int e : p->cuts) cd2[e] = 1;
    PathGraph pg2 = make_pg(g.n, g.eu, g.ev, cd2);
    s = path_auto(pg2, o, p->order, p->score, pops, p->rank_used);
    p->pops += pops;
    if (s != TN_OK) return s;
  } else {
    s = choose_cuts(g, o, dims, o.n_cuts, limit, p->cuts, p->order, p->score, p->pops, p->rank_used);
    if (s != TN_OK) return s;
  }
  if (two_layers && !o.no_merge) join_paths(p);
  s = compile_plan(p);
  if (s != TN_OK) return s;
  const double budget = o.mem_budget_bytes > 0 ? o.mem_budget_bytes : 8.0 * (1ull << 30);
  for (int kind = 0; kind < 2; ++kind) {
    // as many whole bitstrings (all slices) as fit; else one bitstring and groups of its slices
    const int64_t grid_cap = 1LL << 40;   // items * maxT bound keeping every launch grid < 2^31 CTAs
    // the workspace is a fixed part (the merged ket, flags) plus a part per bitstring
    const int64_t fixed = plan_ws_bytes(p, kind, 0, p->n_slices);
    const int64_t per = plan_ws_bytes(p, kind, 1, p->n_slices) - fixed;
    int64_t ch = (int64_t)std::floor((budget - (double)fixed) / (double)per);
    ch = std::min<int64_t>(ch, 1 << 16);
    while (ch > 1 && ch * p->n_slices * std::max<int64_t>(p->maxT, 1) >= grid_cap) ch /= 2;
    int64_t sc = p->n_slices;
    if (ch < 1) {
      ch = 1;
      const int64_t per_slice = plan_ws_bytes(p, kind, 1, 2) - plan_ws_bytes(p, kind, 1, 1);
      sc = (int64_t)std::floor((budget - (double)plan_ws_bytes(p, kind, 1, 0)) / (double)per_slice);
      sc = std::max<int64_t>(1, std::min(sc, p->n_slices));
      while (sc > 1 && sc * std::max<int64_t>(p->maxT, 1) >= grid_cap) sc /= 2;
    }
    p->chunk[kind] = (int)ch;
    p->slice_chunk[kind] = sc;
    p->ws_bytes[kind] = plan_ws_bytes(p, kind, ch, sc);
  }
  return TN_OK;
}

extern "C" tn_status tn_path(tn_circuit *c, const tn_path_opts *opts, tn_plan **out, tn_plan_info *info) {
  if (!c || !out) return tn_fail(TN_ERR_ARG, "tn_path: NULL argument");
  *out = nullptr;
  if (!c->evolved) return tn_fail(TN_ERR_STATE, "tn_path: call tn_evolve_two_sided first");
  const tn_path_opts o = opts ? *opts : tn_default_opts();
  tn_plan *p = new tn_plan();
  tn_status s = no_throw("tn_path", [&] { return plan_host(c, o, p); });
  if (s != TN_OK) { delete p; return s; }
  const bool two_layers = o.layers == 2;
  // upload tables
  cudaStream_t st = 0;
  s = c->mem.ensure(p->tab_dev, std::max<size_t>(p->tab_host.size(), 1) * sizeof(int32_t), st);
  if (s != TN_OK) { delete p; return s; }
  cudaError_t ce = cudaMemcpy(p->tab_dev.p, p->tab_host.data(), p->tab_host.size() * sizeof(int32_t),
                              cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    c->mem.release(p->tab_dev);
    delete p;
    return tn_fail(TN_ERR_CUDA, "table upload: %s", cudaGetErrorString(ce));
  }
  if (two_layers) {   // the unit operand [1, 0]: complex128 at byte 0, complex64 at byte 32
    s = c->mem.ensure(p->unit_dev, 64, st);
    if (s != TN_OK) {
      c->mem.release(p->tab_dev);
      delete p;
      return s;
    }
    uint8_t u[64] = {0};
    const double one = 1.0;
    const float onef = 1.0f;
    std::memcpy(u, &one, sizeof one);
    std::memcpy(u + 32, &onef, sizeof onef);
    ce = cudaMemcpy(p->unit_dev.p, u, sizeof u, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
      c->mem.release(p->unit_dev);
      c->mem.release(p->tab_dev);
      delete p;
      return tn_fail(TN_ERR_CUDA, "unit operand upload: %s", cudaGetErrorString(ce));
    }
  }
  fill_info(p, info);
  *out = p;
  return TN_OK;
}

// A host copy of circuit c with the structural gate programs of (split, chi, cutoff) and no
// device state: what tn_path compiles, without the rank probe and the ket evolution.
static tn_status host_programs(const tn_circuit *c, int32_t split_cycle, int32_t chi_max, double cutoff_rel,
                               tn_circuit &h) {
  if (split_cycle < 0 || chi_max < 0 || !(cutoff_rel >= 0) || cutoff_rel >= 1)
    return tn_fail(TN_ERR_ARG, "bad split/chi/cutoff");
  h.n = c->n;
  h.ne = c->ne;
  h.max_deg = c->max_deg;
  h.eu = c->eu;
  h.ev = c->ev;
  h.legs = c->legs;
  h.gates = c->gates;
  h.compress = h.built_compress = c->compress;
  std::vector<const tn_gate *> g1, g2;
  for (const auto &g : h.gates) (g.cycle <= split_cycle ? g1 : g2).push_back(&g);
  std::reverse(g2.begin(), g2.end());
  build_half(&h, g1, false, chi_max, cutoff_rel, h.ket);
  build_half(&h, g2, true, chi_max, cutoff_rel, h.bra);
  h.split = split_cycle;
  h.chi = chi_max;
  h.cutoff = cutoff_rel;
  h.evolved = true;
  return TN_OK;
}

static tn_status plan_estimate_impl(const tn_circuit *c, int32_t split_cycle, int32_t chi_max, double cutoff_rel,
                                    const tn_path_opts *opts, tn_plan_info *info) {
  tn_circuit h;
  tn_status s = host_programs(c, split_cycle, chi_max, cutoff_rel, h);
  if (s != TN_OK) return s;
  const tn_path_opts o = opts ? *opts : tn_default_opts();
  tn_plan p;
  if ((s = plan_host(&h, o, &p)) != TN_OK) return s;
  fill_info(&p, info);
  return TN_OK;
}

extern "C" tn_status tn_plan_estimate(const tn_circuit *c, int32_t split_cycle, int32_t chi_max, double cutoff_rel,
                                      const tn_path_opts *opts, tn_plan_info *info) {
  if (!c || !info) return tn_fail(TN_ERR_ARG, "tn_plan_estimate: NULL argument");
  return no_throw("tn_plan_estimate", [&] { return plan_estimate_impl(c, split_cycle, chi_max, cutoff_rel, opts, info); });
}

static_assert(TN_PLAN_MAXREST == TN_MAXREST, "rest-leg limit of the inspection layout");

static tn_status plan_inspect_impl(const tn_circuit *c, int32_t split_cycle, int32_t chi_max, double cutoff_rel,
                                   const tn_path_opts *opts, int64_t *layout, int64_t *steps, int32_t *tables,
                                   int64_t *n_steps, int64_t *n_tables) {
  tn_circuit h;
  tn_status s = host_programs(c, split_cycle, chi_max, cutoff_rel, h);
  if (s != TN_OK) return s;
  const tn_path_opts o = opts ? *opts : tn_default_opts();
  tn_plan p;
  if ((s = plan_host(&h, o, &p)) != TN_OK) return s;
  *n_steps = (int64_t)p.steps.size();
  *n_tables = (int64_t)p.tab_host.size();
  if (layout) {
    layout[0] = p.maxT;
    layout[1] = p.n_slices;
    layout[2] = (int64_t)p.steps.size();
    layout[3] = p.net.ket_elems;
    layout[4] = p.net.bra_elems;
    layout[5] = p.net.merged() ? 1 : 0;
    layout[6] = h.ket.item_elems;
    layout[7] = h.bra.item_elems;
    for (int q = 0; q < h.n; ++q) {
      layout[8 + 2 * q] = h.ket.node_off[q];
      layout[9 + 2 * q] = h.bra.node_off[q];
    }
    const int64_t b = 8 + 2 * (int64_t)h.n;
    for (int e = 0; e < h.ne; ++e) {
      layout[b + 2 * e] = h.ket.dims[e];
      layout[b + 2 * e + 1] = h.bra.dims[e];
    }
  }
  if (steps)
    for (size_t j = 0; j < p.steps.size(); ++j) {
      const StepParams &q = p.steps[j];
      int64_t *d = steps + (int64_t)j * TN_STEP_DESC_LEN;
      const int64_t head[17] = {q.M, q.K, q.N, p.step_layer[j], q.n_rest, q.ket_off, q.ket_sig, q.bra_off,
                                q.bra_sig, q.phys, q.t_ocol, q.t_bka, q.t_bkb, q.t_bna, q.t_bnb, q.t_sa, q.t_sb};
      for (int t = 0; t < 17; ++t) d[t] = head[t];
      for (int r = 0; r < TN_MAXREST; ++r) {
        d[17 + r] = r < q.n_rest ? q.rest_dim[r] : 0;
        d[17 + TN_MAXREST + r] = r < q.n_rest ? q.rest_ostride[r] : 0;
      }
    }
  if (tables) std::memcpy(tables, p.tab_host.data(), p.tab_host.size() * sizeof(int32_t));
  return TN_OK;
}

extern "C" tn_status tn_plan_inspect(const tn_circuit *c, int32_t split_cycle, int32_t chi_max, double cutoff_rel,
                                     const tn_path_opts *opts, int64_t *layout, int64_t *steps, int32_t *tables,
                                     int64_t *n_steps, int64_t *n_tables) {
  if (!c || !n_steps || !n_tables) return tn_fail(TN_ERR_ARG, "tn_plan_inspect: NULL argument");
  return no_throw("tn_plan_inspect", [&] {
    return plan_inspect_impl(c, split_cycle, chi_max, cutoff_rel, opts, layout, steps, tables, n_steps, n_tables);
  });
}

static_assert(TN_PROG_ENTRY_LEN == 16 && TN_PROG_MAT_LEN == 66, "gate program inspection layout");

static tn_status program_inspect_impl(const tn_circuit *c, int32_t split_cycle, int32_t chi_max, double cutoff_rel,
                                      int32_t side, int64_t *entries, double *mats, int64_t *n_entries) {
  tn_circuit h;
  tn_status s = host_programs(c, split_cycle, chi_max, cutoff_rel, h);
  if (s != TN_OK) return s;
  const Half &hf = side ? h.bra : h.ket;
  *n_entries = (int64_t)hf.seq.size();
  if (!entries || !mats) return TN_OK;
  for (size_t j = 0; j < hf.seq.size(); ++j) {
    int64_t *e = entries + j * TN_PROG_ENTRY_LEN;
    double *m = mats + j * TN_PROG_MAT_LEN;
    for (int i = 0; i < TN_PROG_ENTRY_LEN; ++i) e[i] = -1;
    for (int i = 0; i < TN_PROG_MAT_LEN; ++i) m[i] = 0;
    const int op = hf.seq[j].first, idx = hf.seq[j].second;
    e[0] = op;
    if (op == 2) {
      const GateParams &g = hf.gp[idx];
      const int k = hf.gate_nodes[idx].first, l = hf.gate_nodes[idx].second;
      const int64_t v[16] = {2, k, l, h.legs[k][g.pk], g.sv_is_k, g.din, g.chi_o, g.n, g.dout, g.m_k, g.m_l,
                             g.pk, g.pl, g.off_k, g.off_l, g.id};
      for (int i = 0; i < 16; ++i) e[i] = v[i];
      for (int i = 0; i < 16; ++i) {
        m[2 * i] = g.P[i].x;
        m[2 * i + 1] = g.P[i].y;
        m[32 + 2 * i] = g.Q[i].x;
        m[32 + 2 * i + 1] = g.Q[i].y;
      }
      m[64] = g.cutoff;
    } else {
      const Apply1Params &a = hf.ap[idx];
      e[1] = hf.ap_node[idx];
      e[13] = a.off;
      for (int i = 0; i < 4; ++i) {
        m[2 * i] = a.u[i].x;
        m[2 * i + 1] = a.u[i].y;
      }
    }
  }
  return TN_OK;
}

extern "C" tn_status tn_program_inspect(const tn_circuit *c, int32_t split_cycle, int32_t chi_max, double cutoff_rel,
                                        int32_t side, int64_t *entries, double *mats, int64_t *n_entries) {
  if (!c || !n_entries || (side != 0 && side != 1)) return tn_fail(TN_ERR_ARG, "tn_program_inspect: bad argument");
  return no_throw("tn_program_inspect", [&] {
    return program_inspect_impl(c, split_cycle, chi_max, cutoff_rel, side, entries, mats, n_entries);
  });
}

extern "C" tn_status tn_set_svd_sweeps(tn_circuit *c, int32_t max_sweeps) {
  if (!c) return tn_fail(TN_ERR_ARG, "tn_set_svd_sweeps: NULL circuit");
  if (max_sweeps < 0 || max_sweeps > 1000) return tn_fail(TN_ERR_ARG, "tn_set_svd_sweeps: %d outside [0, 1000]", max_sweeps);
  c->max_sweeps = c->ket.max_sweeps = c->bra.max_sweeps = max_sweeps;
  return TN_OK;
}

extern "C" tn_status tn_set_compression(tn_circuit *c, int32_t mode) {
  if (!c) return tn_fail(TN_ERR_ARG, "tn_set_compression: NULL circuit");
  if (mode != TN_COMPRESS_ONE_SIDED && mode != TN_COMPRESS_TWO_SIDED)
    return tn_fail(TN_ERR_ARG, "tn_set_compression: unknown mode %d", (int)mode);
  c->compress = mode;
  return TN_OK;
}

extern "C" tn_status tn_plan_details(const tn_plan *p, int32_t *order, int32_t *cuts, int64_t *steps) {
  if (!p) return tn_fail(TN_ERR_ARG, "tn_plan_details: NULL plan");
  if (order) {
    if (!p->net.layer.empty())
      for (int j = 0; j < p->net.n; ++j) order[j] = p->net.dl_id[p->order[j]];
    else
      for (int j = 0; j < p->c->n; ++j) order[j] = j < p->net.n ? p->net.rep[p->order[j]] : -1;
  }
  if (cuts)
    for (size_t j = 0; j < p->cuts.size(); ++j) cuts[j] = p->net.eid[p->cuts[j]];
  if (steps)
    for (size_t j = 1; j < p->step_mkn.size(); ++j)
      for (int t = 0; t < 3; ++t) steps[3 * (j - 1) + t] = p->step_mkn[j][t];
  return TN_OK;
}

// ---------------------------------------------------------------------------
// tn_amplitudes
// ---------------------------------------------------------------------------
void ws_release(DevMem &mem, Workspace &w) {
  if (w.fixed) {   // not the library's memory
    w = Workspace();
    return;
  }
  mem.release(w.bits);
  mem.release(w.bra64);
  mem.release(w.bra32);
  mem.release(w.gwork);
  mem.release(w.t0);
  mem.release(w.t1);
  mem.release(w.res);
  mem.release(w.err);
  mem.release(w.cbuf);
  mem.release(w.ket64);
  mem.release(w.ket32);
}

// Byte sizes of a workspace's buffers for `ch` bitstrings of `sc` slices each (the FP64 form when
// kind == 0, the complex64 / tensor-core forms when kind == 1).
WsSizes ws_sizes(const tn_plan *p, int kind, int64_t ch, int64_t sc) {
  const tn_circuit *c = p->c;
  const int words = (c->n + 63) / 64;
  WsSizes z;
  z.b[WS_BITS] = ch * words * 8;
  z.b[WS_BRA64] = ch * p->net.bra_elems * 16;
  z.b[WS_BRA32] = kind ? ch * p->net.bra_elems * 8 : 0;
  z.b[WS_KET64] = p->net.merged() ? p->net.ket_elems * 16 : 0;
  z.b[WS_KET32] = p->net.merged() && kind ? p->net.ket_elems * 8 : 0;
  z.b[WS_GWORK] = ch * std::max<int64_t>(c->bra.max_work, 1) * 16;
  z.b[WS_T0] = z.b[WS_T1] = ch * sc * p->maxT * (kind ? 12 : 16);
  z.b[WS_CBUF] = kind ? ch * sc * p->maxKN * 24 : 0;
  z.b[WS_RES] = ch * 16;
  z.b[WS_ERR] = 64;
  z.total = 0;
  for (int i = 0; i < WS_NBUF; ++i) z.total += (z.b[i] + 255) & ~int64_t(255);
  return z;
}

static Buf *ws_buf(Workspace &w, int i) {
  Buf *t[WS_NBUF] = {&w.bits, &w.bra64, &w.bra32, &w.ket64, &w.ket32, &w.gwork, &w.t0, &w.t1, &w.cbuf, &w.res, &w.err};
  return t[i];
}

void ws_carve(Workspace &w, void *base, const WsSizes &z, int64_t ch, int64_t sc, cudaStream_t st) {
  unsigned char *cur = static_cast<unsigned char *>(base);
  for (int i = 0; i < WS_NBUF; ++i) {
    Buf &b = *ws_buf(w, i);
    b.p = z.b[i] ? cur : nullptr;
    b.bytes = (size_t)z.b[i];
    b.stream = st;
    cur += (z.b[i] + 255) & ~int64_t(255);
  }
  w.chunk = (int)ch;
  w.slice_chunk = sc;
}

tn_status ws_ensure_sized(tn_plan *p, Workspace &w, int kind, int64_t ch, int64_t sc, cudaStream_t st) {
  DevMem &mem = p->c->mem;
  const WsSizes z = ws_sizes(p, kind, ch, sc);
  if (w.fixed) {   // caller memory: it holds these sizes or the call is refused, never allocated
    for (int i = 0; i < WS_NBUF; ++i)
      if ((size_t)z.b[i] > ws_buf(w, i)->bytes)
        return tn_fail(TN_ERR_OOM, "workspace in fixed memory is too small for %lld bitstrings", (long long)ch);
    return TN_OK;
  }
  for (int i = 0; i < WS_NBUF; ++i) {
    tn_status s = mem.ensure(*ws_buf(w, i), (size_t)z.b[i], st);
    if (s != TN_OK) return s;
  }
  w.chunk = (int)ch;
  w.slice_chunk = sc;
  return TN_OK;
}

tn_status ws_ensure(tn_plan *p, Workspace &w, int kind, cudaStream_t st) {
  return ws_ensure_sized(p, w, kind, p->chunk[kind], p->slice_chunk[kind], st);
}

bool step_kernel_ok(const StepParams &s, tn_precision prec, int k) {
  // a double-layer step (one tensor and the unit operand, a zero physical stride) never uses a
  // kernel that builds the operand from node tensors staged in shared memory
  if ((s.ket_sig == 0 || s.bra_sig == 0) && sk_is_tma(k) && sk_tma_bmode(k) == 1) return false;
  if (k < SK_TC) return simt_variant_ok(s, k, prec == TN_FP64);
  if (k == SK_TC) return prec != TN_FP64 && prec != TN_FP32 && prec != TN_BF16X6 && tc_step_supported(s);
  if (!sk_is_tma(k)) return false;
  if (prec != TN_BF16X6 || !tma_step_supported(s)) return false;
  // the persistent form keeps three order-0 accumulators at either tile width (TMEM holds two
  // accumulator sets at 64 columns), so it takes the short-K rule of the 128-column tile
  if (sk_tma_persist(k) && s.K >= TN_TMA_LONG_K) return false;
  return sk_tma_bn(k) != 128 || (2 * s.N >= 128 && s.K < TN_TMA_LONG_K);
}

// The tuned kernels of the plan for this precision, else the shape heuristic: TMA-fed tcgen05 for
// BF16x6, the in-kernel split tcgen05 kernel for the other tensor-core forms, SIMT elsewhere.
std::vector<int> step_kernels(const tn_plan *p, tn_precision prec) {
  const std::vector<int> &t = p->tune[prec];
  if (t.size() == p->steps.size()) return t;
  std::vector<int> k(p->steps.size(), SIMT_AUTO);
  for (size_t j = 1; j < p->steps.size(); ++j) {
    if (prec == TN_BF16X6 && step_kernel_ok(p->steps[j], prec, SK_TMAC)) k[j] = SK_TMAC;
    else if (step_kernel_ok(p->steps[j], prec, SK_TC)) k[j] = SK_TC;
  }
  return k;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The intermediate's output format: bf16 pieces when the consuming step's kernel reads them (the
// TMA-fed kernels but the complex64-A one), else complex.
static OutDesc out_desc(void *buf, const std::vector<int> &ks, size_t consumer, int64_t plane_u32) {
  OutDesc o;
  o.p = buf;
  o.fmt = (consumer < ks.size() && sk_reads_pieces(ks[consumer])) ? 1 : 0;
  o.plane_u32 = plane_u32;
  return o;
}

// One contraction step j of a slice group with kernel k, with the overlap formation that kernel
// needs as a separate pass (tcgen05 paths); SIMT steps form the overlap tensor on the fly.
cudaError_t enqueue_step(const tn_plan *p, const Workspace &w, size_t j, int k, tn_precision prec,
                         const ContractArgs &a, const void *ket, const void *bra, const void *tin, void *tout,
                         const OutDesc &od, cudaStream_t st) {
  const StepParams &sp = p->steps[j];
  const int kind = prec == TN_FP64 ? 0 : 1;
  const double el = kind ? 8.0 : 16.0;
  const double items = (double)a.items;
  const double by = el * items * ((double)sp.M * sp.K + (double)sp.M * sp.N);
  const double fl = 8.0 * items * (double)sp.M * sp.K * sp.N;
  const int64_t cap = (int64_t)w.chunk * w.slice_chunk;
  if (prec == TN_FP64) {
    ProfScope ps(k == SIMT_BOX ? "contract_step_fp64_box" : "contract_step_fp64", st, by, fl);
    return launch_step<double>(sp, a, ket, bra, tin, od, st, k);
  }
  if (k < SK_TC) {
    ProfScope ps(k == SIMT_BOX ? (prec == TN_FP32 ? "contract_step_fp32_box" : "contract_step_fp32_box_tc_fallback")
                               : (prec == TN_FP32 ? "contract_step_fp32" : "contract_step_fp32_tc_fallback"),
                 st, by, fl);
    return launch_step<float>(sp, a, ket, bra, tin, od, st, k);
  }
  if (k == SK_TC) {
    {
      ProfScope ps("overlap_form_c64", st, 8.0 * items * (double)sp.K * sp.N, 16.0 * items * (double)sp.K * sp.N);
      cudaError_t e = launch_form_c(sp, a, (const float2 *)ket, (const float2 *)bra, (float2 *)w.cbuf.p, p->maxKN, st);
      if (e != cudaSuccess) return e;
    }
    ProfScope ps("contract_step_tcgen05", st, by + 8.0 * items * (double)sp.K * sp.N, fl);
    return launch_step_tc((int)prec, sp, a, (const float2 *)w.cbuf.p, p->maxKN, (const float2 *)tin, (float2 *)tout,
                          (int *)w.err.p + 1, st);
  }
  Pieces A, B;
  A.base = const_cast<void *>(tin);
  A.item_elems = 2 * p->maxT;
  A.plane_elems = cap * A.item_elems;
  B.base = w.cbuf.p;
  B.item_elems = 4 * p->maxKN;
  B.plane_elems = cap * B.item_elems;
  const double out_b = (od.fmt ? 12.0 : 8.0) * (double)sp.M * sp.N;
  if (sk_tma_bmode(k) == 1) {
    // algorithmic bytes: A pieces read, output written (B is built on chip from the node tensors)
    ProfScope ps("contract_step_tcgen05_tma_buildb", st, items * (12.0 * (double)sp.M * sp.K + out_b), fl);
    return launch_step_tma(sp, a, A, B, od, (int *)w.err.p + 1, st, sk_tma_bn(k), (const float2 *)ket,
                           (const float2 *)bra);
  }
  if (sk_tma_bmode(k) == 2) {
    // a ket tensor's overlap operand does not depend on the bitstring, only on the slice: items
    // 0 .. n_slices - 1 (the first bitstring's) hold every distinct copy, formed once
    const bool shared = j < p->step_layer.size() && p->step_layer[j] == 1;
    const int64_t c_items = shared ? a.n_slices : a.items;
    {
      ContractArgs af = a;
      af.items = c_items;
      ProfScope ps("overlap_form_c64", st, 8.0 * c_items * (double)sp.K * sp.N, 16.0 * c_items * (double)sp.K * sp.N);
      cudaError_t e = launch_form_c(sp, af, (const float2 *)ket, (const float2 *)bra, (float2 *)w.cbuf.p, p->maxKN, st);
      if (e != cudaSuccess) return e;
    }
    if (sk_tma_c64a(k)) {
      // algorithmic bytes: A and the overlap tensor read as complex64, output written
      ProfScope ps("contract_step_tcgen05_tma_persist_c64a", st,
                   items * (8.0 * (double)sp.M * sp.K + out_b) + 8.0 * c_items * (double)sp.K * sp.N, fl);
      return launch_step_tma_persistent(sp, a, A, B, od, (int *)w.err.p + 1, st, sk_tma_bn(k),
                                        (const float2 *)w.cbuf.p, p->maxKN, c_items, (const float2 *)tin);
    }
    // algorithmic bytes: A pieces and the complex64 overlap tensor read, output written
    const double by_c = items * (12.0 * (double)sp.M * sp.K + out_b) + 8.0 * c_items * (double)sp.K * sp.N;
    if (sk_tma_persist(k)) {
      ProfScope ps("contract_step_tcgen05_tma_persist", st, by_c, fl);
      return launch_step_tma_persistent(sp, a, A, B, od, (int *)w.err.p + 1, st, sk_tma_bn(k),
                                        (const float2 *)w.cbuf.p, p->maxKN, c_items);
    }
    ProfScope ps("contract_step_tcgen05_tma", st, by_c, fl);
    return launch_step_tma(sp, a, A, B, od, (int *)w.err.p + 1, st, sk_tma_bn(k), nullptr, nullptr,
                           (const float2 *)w.cbuf.p, p->maxKN, c_items);
  }
  if (sk_tma_persist(k)) {
    // B pieces formed in HBM (once per slice for a ket tensor) and loaded by TMA
    const bool shared = j < p->step_layer.size() && p->step_layer[j] == 1;
    const int64_t c_items = shared ? a.n_slices : a.items;
    {
      ContractArgs af = a;
      af.items = c_items;
      ProfScope ps("overlap_form_bf16_pieces", st, 24.0 * c_items * (double)sp.K * sp.N,
                   16.0 * c_items * (double)sp.K * sp.N);
      cudaError_t e = launch_form_b_pieces(sp, af, (const float2 *)ket, (const float2 *)bra, B, st);
      if (e != cudaSuccess) return e;
    }
    const bool c64a = sk_tma_c64a(k);
    const double by_p = items * ((c64a ? 8.0 : 12.0) * (double)sp.M * sp.K + out_b) + 24.0 * c_items * (double)sp.K * sp.N;
    ProfScope ps(c64a ? "contract_step_tcgen05_tma_persist_c64a_loadb" : "contract_step_tcgen05_tma_persist_loadb", st,
                 by_p, fl);
    return launch_step_tma_persistent(sp, a, A, B, od, (int *)w.err.p + 1, st, sk_tma_bn(k), nullptr, 0, c_items,
                                      c64a ? (const float2 *)tin : nullptr);
  }
  {
    ProfScope ps("overlap_form_bf16_pieces", st, 24.0 * items * (double)sp.K * sp.N, 16.0 * items * (double)sp.K * sp.N);
    cudaError_t e = launch_form_b_pieces(sp, a, (const float2 *)ket, (const float2 *)bra, B, st);
    if (e != cudaSuccess) return e;
  }
  // algorithmic bytes of the step in its operand format: A and B pieces read, output written
  ProfScope ps("contract_step_tcgen05_tma_loadb", st, items * (12.0 * (double)sp.M * sp.K + 24.0 * (double)sp.K * sp.N + out_b),
               fl);
  return launch_step_tma(sp, a, A, B, od, (int *)w.err.p + 1, st, sk_tma_bn(k));
}

void step_operands(const tn_plan *p, size_t j, int kind, const void *ket, const void *bra, const ContractArgs &a,
                   const void *&kj, const void *&bj, ContractArgs &aj) {
  kj = ket;
  bj = bra;
  aj = a;
  const int lay = j < p->step_layer.size() ? p->step_layer[j] : 0;
  if (lay == 0) return;
  // double-layer step: the slot that is not the absorbed tensor's reads the unit operand
  const void *unit = (const uint8_t *)p->unit_dev.p + (kind ? 32 : 0);
  if (lay == 1) {
    bj = unit;
    aj.bra_stride = 0;
  } else {
    kj = unit;
  }
}

// Bra evolution and contraction of nb <= w.chunk bitstrings already on the device, amplitudes to
// res_dev (nb complex128 on the device). Stream-ordered work only (no allocation, no host
// synchronisation), so it can also be captured into a CUDA graph. The error words in w.err are
// set, never cleared, here.
tn_status enqueue_chunk(tn_plan *p, Workspace &w, const uint64_t *bits_dev, int64_t nb, tn_precision prec,
                        const std::vector<int> &ks, double2 *res_dev, cudaStream_t st, int64_t slice_begin,
                        int64_t slice_end) {
  tn_circuit *c = p->c;
  const int kind = prec == TN_FP64 ? 0 : 1;
  const int words = (c->n + 63) / 64;
  const int64_t S = slice_end < 0 ? p->n_slices : std::min<int64_t>(slice_end, p->n_slices);
  const int64_t S0 = std::max<int64_t>(slice_begin, 0);
  if (S0 >= S) {   // no slice: the partial sum is zero
    CUDA_TRY(cudaMemsetAsync(res_dev, 0, nb * sizeof(double2), st));
    return TN_OK;
  }
  const Net &g = p->net;
  tn_status s = run_half(c->bra, c->n, (double2 *)w.bra64.p, (int)nb, (const int64_t *)c->bra_off_dev.p, bits_dev,
                         words, (double2 *)w.gwork.p, (int *)w.err.p, st, nullptr, nullptr, g.bra_elems);
  if (s != TN_OK) return s;
  if (g.merged()) {
    // merged nodes: the ket's once per batch (one item) in FP64; the bra's per bitstring, in FP64
    // for the FP64 form and in FP32 after the conversion below for the complex64 forms (whose
    // contraction carries FP32-level products anyway; FP64 arithmetic runs at a small fraction of
    // the FP32 rate)
    CUDA_TRY(cudaMemcpyAsync(w.ket64.p, c->ket_dev.p, c->ket.item_elems * sizeof(double2), cudaMemcpyDeviceToDevice,
                             st));
    for (const MergeParams &m : g.mk) {
      ProfScope ps("merge_nodes_fp64", st, 16.0 * (m.out_size + m.out_size * m.da), 8.0 * m.out_size * m.da);
      CUDA_TRY(launch_merge(m, (double2 *)w.ket64.p, g.ket_elems, 1, st));
    }
    if (!kind)
      for (const MergeParams &m : g.mb) {
        ProfScope ps("merge_nodes_fp64", st, 16.0 * nb * (m.out_size + m.out_size * m.da),
                     8.0 * nb * m.out_size * m.da);
        CUDA_TRY(launch_merge(m, (double2 *)w.bra64.p, g.bra_elems, nb, st));
      }
    if (kind) CUDA_TRY(launch_to_c64((const double2 *)w.ket64.p, (float2 *)w.ket32.p, g.ket_elems, st));
  }
  const void *ket = g.merged() ? (kind ? w.ket32.p : w.ket64.p) : (kind ? c->ket_c64.p : c->ket_dev.p);
  const void *bra = w.bra64.p;
  if (kind) {
    {
      ProfScope ps("to_c64", st, 24.0 * nb * g.bra_elems, 0);
      CUDA_TRY(launch_to_c64((const double2 *)w.bra64.p, (float2 *)w.bra32.p, nb * g.bra_elems, st));
    }
    bra = w.bra32.p;
    for (const MergeParams &m : g.mb) {
      ProfScope ps("merge_nodes_fp32", st, 8.0 * nb * (m.out_size + m.out_size * m.da), 8.0 * nb * m.out_size * m.da);
      CUDA_TRY(launch_merge(m, (float2 *)w.bra32.p, g.bra_elems, nb, st));
    }
  }
  const size_t nsteps = p->steps.size();
  const int64_t cap = (int64_t)w.chunk * w.slice_chunk;     // items the buffers hold
  auto operands = [&](size_t j, const ContractArgs &a, const void *&kj, const void *&bj, ContractArgs &aj) {
    step_operands(p, j, kind, ket, bra, a, kj, bj, aj);
  };
  for (int64_t s0 = S0; s0 < S; s0 += w.slice_chunk) {
    const int64_t sg = std::min<int64_t>(w.slice_chunk, S - s0);
    ContractArgs a;
    a.tab = (const int32_t *)p->tab_dev.p;
    a.n_slices = sg;
    a.slice0 = s0;
    a.items = nb * sg;
    a.t_stride = p->maxT;
    a.bra_stride = g.bra_elems;
    void *tin = w.t0.p, *tout = w.t1.p;
    const double el = kind ? 8.0 : 16.0;
    const void *kj, *bj;
    ContractArgs aj;
    {
      ProfScope ps(kind ? "overlap_form_c64" : "overlap_form_c128", st, el * a.items * p->steps[0].N, 0);
      const OutDesc od = out_desc(tin, ks, 1, cap * p->maxT);
      operands(0, a, kj, bj, aj);
      if (kind) CUDA_TRY(launch_form<float>(p->steps[0], aj, kj, bj, od, st));
      else CUDA_TRY(launch_form<double>(p->steps[0], aj, kj, bj, od, st));
    }
    for (size_t j = 1; j < nsteps; ++j) {
      const ProfStep pst((int)j - 1);   // the index of the step in the plan's public lists
      operands(j, a, kj, bj, aj);
      CUDA_TRY(enqueue_step(p, w, j, ks[j], prec, aj, kj, bj, tin, tout,
                            out_desc(tout, ks, j + 1, cap * p->maxT), st));
      std::swap(tin, tout);
    }
    {
      ProfScope ps("slice_sum_fp64", st, (el * sg + 16.0) * nb, 0);
      if (kind) CUDA_TRY(launch_slice_sum<float>(tin, p->maxT, nb, sg, s0 > S0, res_dev, st));
      else CUDA_TRY(launch_slice_sum<double>(tin, p->maxT, nb, sg, s0 > S0, res_dev, st));
    }
  }
  return TN_OK;
}

tn_status check_err_words(const int *err) {
  if (err[0])
    return tn_fail(TN_ERR_TIMEOUT, "Jacobi SVD did not converge within its sweep limit (bra half, gate %d)", err[0] - 1);
  if (err[1]) return tn_fail(TN_ERR_TIMEOUT, "tensor-core GEMM: a bounded pipeline wait expired (code %d)", err[1]);
  return TN_OK;
}

tn_status run_amplitudes(tn_plan *p, Workspace &w, const uint64_t *bits, int64_t n, tn_precision prec,
                         tn_c128 *out, cudaStream_t st, int64_t slice_begin, int64_t slice_end) {
  tn_circuit *c = p->c;
  if (p->generation != c->generation) return tn_fail(TN_ERR_STATE, "plan is stale: the circuit was re-evolved");
  if (prec < TN_FP64 || prec > TN_TF32X6) return tn_fail(TN_ERR_ARG, "unknown precision %d", (int)prec);
  if (n == 0) return TN_OK;
  if (n < 0 || !bits || !out) return tn_fail(TN_ERR_ARG, "tn_amplitudes: bad arguments");
  const int kind = prec == TN_FP64 ? 0 : 1;
  // buffers for min(n, chunk) bitstrings (they grow when a later call needs more); a fixed
  // workspace runs in its own batch size
  tn_status s = w.fixed ? TN_OK
                        : ws_ensure_sized(p, w, kind, std::min<int64_t>(std::max<int64_t>(n, w.chunk), p->chunk[kind]),
                                          p->slice_chunk[kind], st);
  if (s != TN_OK) return s;
  const int words = (c->n + 63) / 64;
  const bool bits_dev = is_device_ptr(bits), out_dev = is_device_ptr(out);
  const std::vector<int> ks = step_kernels(p, prec);
  CUDA_TRY(cudaMemsetAsync(w.err.p, 0, 2 * sizeof(int), st));
  for (int64_t start = 0; start < n; start += w.chunk) {
    const int64_t nb = std::min<int64_t>(w.chunk, n - start);
    CUDA_TRY(cudaMemcpyAsync(w.bits.p, bits + start * words, nb * words * 8,
                             bits_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    s = enqueue_chunk(p, w, (const uint64_t *)w.bits.p, nb, prec, ks, (double2 *)w.res.p, st, slice_begin,
                      slice_end);
    if (s != TN_OK) return s;
    CUDA_TRY(cudaMemcpyAsync(out + start, w.res.p, nb * sizeof(tn_c128),
                             out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  int err[2] = {0, 0};
  CUDA_TRY(cudaMemcpyAsync(err, w.err.p, sizeof err, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return check_err_words(err);
}

extern "C" tn_status tn_amplitudes(tn_plan *p, const uint64_t *bits, int64_t n, tn_precision prec, tn_c128 *out,
                                   void *cuda_stream) {
  if (!p) return tn_fail(TN_ERR_ARG, "tn_amplitudes: NULL plan");
  return run_amplitudes(p, p->ws, bits, n, prec, out, (cudaStream_t)cuda_stream);
}

extern "C" tn_status tn_amplitudes_slices(tn_plan *p, const uint64_t *bits, int64_t n, tn_precision prec,
                                          int64_t slice_begin, int64_t slice_end, tn_c128 *out, void *cuda_stream) {
  if (!p) return tn_fail(TN_ERR_ARG, "tn_amplitudes_slices: NULL plan");
  if (slice_begin < 0 || slice_end < slice_begin || slice_end > p->n_slices)
    return tn_fail(TN_ERR_ARG, "tn_amplitudes_slices: slice range [%lld, %lld) outside [0, %lld)",
                   (long long)slice_begin, (long long)slice_end, (long long)p->n_slices);
  return run_amplitudes(p, p->ws, bits, n, prec, out, (cudaStream_t)cuda_stream, slice_begin, slice_end);
}

extern "C" void tn_plan_free(tn_plan *p) {
  if (!p) return;
  cudaDeviceSynchronize();
  ws_release(p->c->mem, p->ws);
  p->c->mem.release(p->tab_dev);
  p->c->mem.release(p->unit_dev);
  delete p;
}
