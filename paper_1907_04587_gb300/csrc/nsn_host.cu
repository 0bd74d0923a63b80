// nsn_host.cu -- host runtime and C ABI of the non-smooth Newton stepper
// (declared in include/nsn.h).  Builds the device layout from the scene,
// owns all device memory, enqueues one time step (Algorithm 1) on the
// context stream and captures it once as a CUDA graph.
#include <cuda.h>   // CUcontext, CUresult (types only)
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "../../include/nsn.h"
#include "nsn_kernels.cuh"
#include "nsn_mlp.cuh"
#include "nsn_mlp_tc.cuh"
#include "nsn_internal.h"
#include "nsn_hostpar.h"

using namespace nsn;

namespace {

// Resident 256-thread blocks of the current device (SMs x threads per SM /
// 256): the cap of every grid and the capacity of the per-block partial sums.
int device_max_blocks() {
  int dev = 0, nsm = 0, thr = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 1;
  if (cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess || thr < BLOCK)
    thr = BLOCK;
  return nsm * (thr / BLOCK);
}

struct HostScene {
  std::vector<int32_t> kind;
  std::vector<float> pos, quat, vel, omega, mass, inertia;
  std::vector<nsn_contact> contacts;
  std::vector<nsn_revolute> joints;
  std::vector<int32_t> jkind;       // per joint: 0 revolute, 1 prismatic
  std::vector<nsn_tet> tets;        // stable Neo-Hookean
  std::vector<nsn_tet> ltets;       // linear Hookean (Sec. 9.2.1)
};

// Bump allocator over one device allocation.
struct Arena {
  char *base = nullptr;
  size_t size = 0, off = 0;
  bool sizing = true;
  template <typename X>
  X *take(size_t n) {
    size_t bytes = ((n ? n : 1) * sizeof(X) + 255) & ~size_t(255);
    X *p = sizing ? nullptr : reinterpret_cast<X *>(base + off);
    off += bytes;
    return p;
  }
};

struct Layout {
  int nr = 0, np = 0, nc = 0, nj = 0, nt = 0, R = 0, Rpair = 0, ER = 0, EV = 0;
  std::vector<int> bmap;            // ABI body id -> encoded (>=0 rigid, <=-2 particle)
  std::vector<int> rig_of, par_of;  // local index -> ABI id
  std::vector<int> eslot, rseg, vseg, re0, re1, te;
  int ni = 0;                       // islands: connected components of bodies through constraints
  std::vector<int> body_isl;        // ABI body id -> island
  std::vector<int> risl, bisl_r, bisl_p;  // island of each row / rigid body / particle
  // Internal order: bodies, contacts, joints and tets sorted by island (stable;
  // islands largest first), so that each island's bodies, entries and rows are
  // contiguous.  The ABI keeps the caller's order; these map internal -> ABI.
  std::vector<int> cperm, jperm, tperm, row_abi;
  // tet blocks of three rows: a Neo-Hookean tet is one block (kind 0); a
  // linear tet is two (kind 1: volumetric and two deviatoric normal-strain
  // modes, kind 2: the three engineering shears); per block (ABI block
  // order) its record and its first ABI row
  std::vector<const nsn_tet *> tb_rec;
  std::vector<int> tb_kind, tb_abi;
  // island-resident CR: per island {c0, nc, j0, nj, b0, nb, e0, ne} (internal
  // order), the eligible islands (rigid bodies, contacts and joints only, at
  // most res_max_rows rows), and the largest eligible island
  std::vector<int> ires;
  std::vector<unsigned char> isres;
  std::vector<unsigned char> isl_rigid;   // 1: the island has no particles and no tets
  int n_res = 0, res_rows = 0, res_ent = 0, res_bod = 0;
  // groups of consecutive eligible islands solved by one thread block
  // ({c0, nc, j0, nj, b0, nb, e0, ne, first slot in gisl, islands} each)
  std::vector<int> gres, gisl, grp_of;
  std::vector<int> isl_order;       // island ids in the internal (rank) order
  int n_streamed = 0;               // islands with rows that the resident CR does not take
  // scratch of the layout build (kept, like the arrays above, across rebuilds:
  // contacts are regenerated every step and their allocations are reused)
  std::vector<int> s_key, s_start, s_rank, s_size, s_cnt, s_fill, s_aux;
  // a new build: every array emptied, its allocation kept
  void reset() {
    for (std::vector<int> *v : {&bmap, &rig_of, &par_of, &eslot, &rseg, &vseg, &re0, &re1, &te, &body_isl, &risl,
                                &bisl_r, &bisl_p, &cperm, &jperm, &tperm, &row_abi, &tb_kind, &tb_abi, &ires, &gres,
                                &gisl, &grp_of, &isl_order})
      v->clear();
    tb_rec.clear();
    isres.clear();
    isl_rigid.clear();
    nr = np = nc = nj = nt = R = Rpair = ER = EV = ni = 0;
    n_res = res_rows = res_ent = res_bod = n_streamed = 0;
  }
};

struct MlpState {
  bool ready = false;
  float *pf = nullptr, *gr = nullptr, *m = nullptr, *v = nullptr;  // FP32 master, gradient, Adam moments
  __nv_bfloat16 *pb = nullptr;                                      // BF16 copy used by the GEMMs
  int adam_t = 0;
  // workspace for up to cap rows (inference chunk or training batch)
  int cap = 0;
  __nv_bfloat16 *xb = nullptr, *a1b = nullptr, *a2b = nullptr, *a3b = nullptr, *dyb = nullptr, *dzb = nullptr;
  float *a1f = nullptr, *a2f = nullptr, *a3f = nullptr, *y = nullptr, *dyf = nullptr, *da = nullptr, *dzf = nullptr,
        *lpart = nullptr;
  // per-contact features and predictions for the learned warm start
  int ncap = 0;
  float *X = nullptr, *Y = nullptr;
  int *err = nullptr;   // set by the inference kernel when a tensor-core wait timed out
};

}  // namespace

// Pinned host staging for the arrays a (re)build writes to the device: chunks
// of page-locked memory kept for the context's lifetime and reused by every
// rebuild (contacts are regenerated every step), so that the host fills no
// fresh pages and the copies run at pinned-memory speed.  A rebuild rewinds
// it; its copies complete before the rebuild returns (stream synchronised).
struct PinnedStage {
  struct Chunk { unsigned char *p; size_t size; };
  std::vector<Chunk> chunks;
  size_t cur = 0, off = 0;
  void rewind() { cur = 0; off = 0; }
  template <typename X>
  X *take(size_t n) {
    const size_t bytes = ((n ? n : 1) * sizeof(X) + 255) & ~size_t(255);
    while (cur < chunks.size() && off + bytes > chunks[cur].size) { cur++; off = 0; }
    if (cur == chunks.size()) {
      Chunk ch{nullptr, std::max<size_t>(bytes, size_t(64) << 20)};
      if (cudaMallocHost(reinterpret_cast<void **>(&ch.p), ch.size) != cudaSuccess) return nullptr;
      chunks.push_back(ch);
      off = 0;
    }
    X *r = reinterpret_cast<X *>(chunks[cur].p + off);
    off += bytes;
    return r;
  }
  void release() {
    for (Chunk &ch : chunks) cudaFreeHost(ch.p);
    chunks.clear();
    rewind();
  }
};

// a contact's identity across contact regenerations: body pair and the bit
// pattern of its point on a (the collider emits corners at fixed body-frame
// points), with the old contact's internal index
struct ContactKeyRec {
  int32_t a, b;
  uint32_t p[3];
  uint32_t n[3];   // compared for contacts with the world only: the plane's normal
  int idx;
};

struct nsn_ctx {
  nsn_config cfg;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  HostScene scene;
  bool dirty = true;
  Layout L;
  void *dmem = nullptr;
  size_t dbytes = 0, dcap = 0;   // bytes in use, bytes allocated
  Dev<float> d32;
  Dev<double> d64;
  int *d_bmap = nullptr;
  float *d_stage = nullptr;  // AoS staging for state transfer (13 floats per body)
  float *d_backup = nullptr; // committed state saved by nsn_linearize
  cudaGraphExec_t graph = nullptr;
  int launches_per_step = 0;  // kernels executed in the last step
  struct Segments { int prefix = 0, head = 0, cr = 0, tail = 0, suffix = 0; } seg;  // kernels per graph segment
  int last_newton_n = 0;     // Newton loop bodies executed in the last step
  int best_restored = 0;     // best_iterate: islands of the last step that returned an earlier iterate
  float tune_ms[3] = {0.f, 0.f, 0.f};  // body-pass times measured by the tuner for 4, 8, 16 lanes
  int forced_lanes = 0;      // nsn_set_body_lanes (0: tuned)
  int tuned_lanes = 0, tuned_nb = -1;   // the tuner's choice and the body count it was made for
  bool linearized = false;
  int lin_buf = 0;           // entry buffer written by the kept linearisation
  int kept_buf = -1;         // entry buffer of the system kept by the last step / linearisation
  int warm_mode = 0;         // NSN_WARM_*
  int warm_friction = 0;     // 1: warm starts also set the friction rows
  int warm_precond = 0;      // 1: the learned start also scales the contacts' Jacobi preconditioner
  MlpState mlp;
  int built_nb = 0;          // bodies present in the current device build
  // previous-step multipliers across a rebuild of the layout (contacts
  // regenerated every step, Sec. 10): the contacts of the built scene, and its
  // joint and tet counts, so that the next build can match them by key
  std::vector<nsn_contact> built_contacts;
  std::vector<nsn_contact> col_rec;   // nsn_collide_and_step: the collider's contacts (reused buffer)
  int built_nj = 0, built_nt = 0;   // joints and tet blocks (3 rows each) of the built scene
  // a rebuild keeps the device's state and previous multipliers on the
  // device: the state in ABI order (13 floats per body, the staging layout)
  // and lam_prev in the old internal row order, with the old internal index
  // of every ABI contact, joint and tet block
  float *keep_state = nullptr;
  size_t keep_state_n = 0;
  void *keep_lam = nullptr;
  size_t keep_lam_bytes = 0;
  bool keep_state_ready = false;
  std::vector<int> old_cinv, old_jinv, old_tinv, lam_map;
  int old_nc = 0, old_Rpair = 0, old_R = 0;
  std::vector<ContactKeyRec> okeys;
  // nsn_collide_and_step: the state handed to the collider (13 floats per
  // body) and its contact buffers (device), with a pinned host copy
  float *col_state = nullptr;
  int col_state_nb = 0;
  int32_t *col_body = nullptr, *col_found = nullptr, *col_found_h = nullptr;
  float *col_f = nullptr, *col_f_h = nullptr;   // pa, pb, n (9), d, mu (2) per contact
  int32_t *col_body_h = nullptr;
  int col_cap = 0;
  int dlog_iters = 0;        // nsn_record_decisions: Newton iterations logged (0: off)
  unsigned char *dlog_buf = nullptr;   // the log on the device (iters x (rows + islands) bytes)
  size_t dlog_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  PinnedStage stage;         // pinned staging of the (re)build's uploads
  std::vector<int> key_end, key_list;      // old contacts bucketed by body a (key matching)
  std::vector<int> key_k, key_cnt;         // scratch of that bucketing
  // host wall time (ms) of the phases of the last rebuild / step, NSN_PHASE_*
  double phase_ms[NSN_PHASES] = {};
  std::string err;
  nsn_stats last{};
};

namespace {
double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
// adds the time since `t0` to a phase and restarts the clock
void phase_tick(nsn_ctx *c, int phase, double &t0) {
  const double t = now_ms();
  c->phase_ms[phase] += t - t0;
  t0 = t;
}
}  // namespace

namespace {

nsn_status fail(nsn_ctx *c, nsn_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CUDA_TRY(c, call)                                                              \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return fail(c, NSN_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

inline int cdiv(long long a, long long b) { return int((a + b - 1) / b); }
inline int clampb(long long n, int max_blk) { return int(std::max(1LL, std::min<long long>(n, max_blk))); }

bool finite_all(const float *p, size_t n) {
  for (size_t i = 0; i < n; i++)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// ------------------------------------------------------------------------------------
// islands: union-find over the bodies of every constraint (the static world is
// not a node); ids follow the order of each island's lowest body, and a row
// belongs to the island of its constraint's bodies

void find_islands(const HostScene &S, Layout &L, int nb) {
  // components on host threads, each rooted at its smallest body
  const long long nc = (long long)S.contacts.size(), nj = (long long)S.joints.size(),
                  nt = (long long)S.tets.size(), nl = (long long)S.ltets.size(), ne = nc + nj + nt + nl;
  std::vector<int> &root = L.s_aux;
  components_min_root(nb, layout_threads(ne), [&](int t, int nth, auto &&unite) {
    const long long e0 = ne * t / nth, e1 = ne * (t + 1) / nth;
    for (long long e = e0; e < e1; e++) {
      if (e < nc) { const auto &r = S.contacts[size_t(e)]; unite(r.body_a, r.body_b); }
      else if (e < nc + nj) { const auto &r = S.joints[size_t(e - nc)]; unite(r.body_a, r.body_b); }
      else {
        const nsn_tet &r = e < nc + nj + nt ? S.tets[size_t(e - nc - nj)] : S.ltets[size_t(e - nc - nj - nt)];
        for (int q = 1; q < 4; q++) unite(r.v[0], r.v[q]);
      }
    }
  }, root);
  std::vector<int> id(nb, -1);
  L.body_isl.assign(nb, 0);
  L.ni = 0;
  for (int i = 0; i < nb; i++) {
    const int r = root[size_t(i)];
    if (id[r] < 0) id[r] = L.ni++;
    L.body_isl[i] = id[r];
  }
}







// ------------------------------------------------------------------------------------
// layout: entries sorted by body (counting sort), rows -> entry ids

nsn_status build_layout(nsn_ctx *c) {
  HostScene &S = c->scene;
  Layout &L = c->L;
  L.reset();
  const int nb = int(S.kind.size());
  find_islands(S, L, nb);
  // Internal island order: largest islands first (ties by id).  Islands that
  // keep iterating after most have stopped are the large ones (long chains),
  // so they cluster and blocks of finished islands are skipped as a whole.
  std::vector<int> &isl_size = L.s_size, &rank = L.s_rank;
  isl_size.assign(L.ni, 0);
  rank.resize(L.ni);
  for (int b = 0; b < nb; b++) isl_size[L.body_isl[b]]++;
  {
    const int maxsz = L.ni ? *std::max_element(isl_size.begin(), isl_size.end()) : 0;
    order_by(L.ni, maxsz + 1, [&](int i) { return maxsz - isl_size[i]; }, L.isl_order, L.s_key, L.s_start);
    for (int k = 0; k < L.ni; k++) rank[L.isl_order[k]] = k;
  }
  // bodies in island order (rigid and particle numbered separately)
  L.bmap.resize(nb);
  order_by(nb, std::max(L.ni, 1), [&](int b) { return rank[L.body_isl[b]]; }, L.s_aux, L.s_key, L.s_start);
  for (int i : L.s_aux) {
    if (S.kind[i] == NSN_RIGID) { L.bmap[i] = L.nr++; L.rig_of.push_back(i); }
    else { L.bmap[i] = -2 - L.np++; L.par_of.push_back(i); }
  }
  L.nc = int(S.contacts.size());
  L.nj = int(S.joints.size());
  L.Rpair = 3 * L.nc + 5 * L.nj;
  for (size_t t = 0; t < S.tets.size(); t++) {
    L.tb_rec.push_back(&S.tets[t]); L.tb_kind.push_back(0); L.tb_abi.push_back(L.Rpair + 3 * int(t));
  }
  const int lrow0 = L.Rpair + 3 * int(S.tets.size());
  for (size_t t = 0; t < S.ltets.size(); t++)
    for (int h = 0; h < 2; h++) {
      L.tb_rec.push_back(&S.ltets[t]); L.tb_kind.push_back(1 + h); L.tb_abi.push_back(lrow0 + 6 * int(t) + 3 * h);
    }
  L.nt = int(L.tb_rec.size());
  L.R = L.Rpair + 3 * L.nt;
  // constraints in island order
  auto isl2 = [&](int a, int b) { return L.body_isl[a >= 0 ? a : b]; };
  const int K = std::max(L.ni, 1);
  order_by(L.nc, K, [&](int i) { return rank[isl2(S.contacts[i].body_a, S.contacts[i].body_b)]; }, L.cperm, L.s_key,
           L.s_start);
  order_by(L.nj, K, [&](int i) { return rank[isl2(S.joints[i].body_a, S.joints[i].body_b)]; }, L.jperm, L.s_key,
           L.s_start);
  order_by(L.nt, K, [&](int i) { return rank[L.body_isl[L.tb_rec[i]->v[0]]]; }, L.tperm, L.s_key, L.s_start);
  L.row_abi.resize(L.R);
  L.risl.resize(L.R);
  {
    const int nth = layout_threads(L.nc);
    parallel_for_threads(nth, [&](int k0) {
      const int c0 = int((long long)L.nc * k0 / nth), c1 = int((long long)L.nc * (k0 + 1) / nth);
      for (int ci = c0; ci < c1; ci++) {
        const auto &r = S.contacts[L.cperm[ci]];
        const int is = isl2(r.body_a, r.body_b);
        for (int k = 0; k < 3; k++) { L.row_abi[3 * ci + k] = 3 * L.cperm[ci] + k; L.risl[3 * ci + k] = is; }
      }
    });
  }
  for (int j = 0; j < L.nj; j++) {
    const auto &r = S.joints[L.jperm[j]];
    for (int k = 0; k < 5; k++) {
      L.row_abi[3 * L.nc + 5 * j + k] = 3 * L.nc + 5 * L.jperm[j] + k;
      L.risl[3 * L.nc + 5 * j + k] = isl2(r.body_a, r.body_b);
    }
  }
  for (int t = 0; t < L.nt; t++)
    for (int k = 0; k < 3; k++) {
      L.row_abi[L.Rpair + 3 * t + k] = L.tb_abi[L.tperm[t]] + k;
      L.risl[L.Rpair + 3 * t + k] = L.body_isl[L.tb_rec[L.tperm[t]]->v[0]];
    }
  L.bisl_r.resize(L.nr);
  L.bisl_p.resize(L.np);
  for (int i = 0; i < L.nr; i++) L.bisl_r[i] = L.body_isl[L.rig_of[i]];
  for (int i = 0; i < L.np; i++) L.bisl_p[i] = L.body_isl[L.par_of[i]];
  // entries: one per (row, side) with a body, sorted by body (rigid, then
  // particle) and within a body by row -- a counting sort over the
  // constraints in row order: each host thread counts the entries of its
  // range of constraints per body, every (body, thread) pair gets its offset
  // (bodies in order, threads in order within a body), and each thread
  // places its range; the result is that of one sequential pass
  const int nbod = L.nr + L.np;
  const long long nitems = (long long)L.nc + L.nj + L.nt;
  const int nth = layout_threads(nitems);
  auto bidx = [&](int enc) { return enc >= 0 ? enc : L.nr + (-enc - 2); };
  // item u: contact u, joint u - nc, tet block u - nc - nj (internal order);
  // fn(row, slot, enc) for each of its entries, rows ascending
  auto visit = [&](long long u, auto &&fn) {
    if (u < L.nc) {
      const int ci = int(u);
      const nsn_contact &r = S.contacts[L.cperm[ci]];
      const int ea = r.body_a >= 0 ? L.bmap[r.body_a] : 0, eb = r.body_b >= 0 ? L.bmap[r.body_b] : 0;
      for (int k = 0; k < 3; k++) {
        if (r.body_a >= 0) fn(3 * ci + k, 0, ea);
        if (r.body_b >= 0) fn(3 * ci + k, 1, eb);
      }
    } else if (u < (long long)L.nc + L.nj) {
      const int j = int(u - L.nc);
      const nsn_revolute &r = S.joints[L.jperm[j]];
      const int ea = r.body_a >= 0 ? L.bmap[r.body_a] : 0, eb = r.body_b >= 0 ? L.bmap[r.body_b] : 0;
      for (int k = 0; k < 5; k++) {
        if (r.body_a >= 0) fn(3 * L.nc + 5 * j + k, 0, ea);
        if (r.body_b >= 0) fn(3 * L.nc + 5 * j + k, 1, eb);
      }
    } else {
      const int tb = int(u - L.nc - L.nj);
      const nsn_tet &r = *L.tb_rec[L.tperm[tb]];
      for (int k = 0; k < 3; k++)
        for (int q = 0; q < 4; q++) fn(L.Rpair + 3 * tb + k, q, L.bmap[r.v[q]]);
    }
  };
  std::vector<int> &cnt = L.s_cnt;            // [body][thread]: counts, then offsets
  cnt.assign(size_t(nth) * nbod, 0);
  parallel_for_threads(nth, [&](int k) {
    int *ck = cnt.data() + k;
    const long long u0 = nitems * k / nth, u1 = nitems * (k + 1) / nth;
    for (long long u = u0; u < u1; u++) visit(u, [&](int, int, int enc) { ck[size_t(bidx(enc)) * nth]++; });
  });
  std::vector<int> &rcnt = L.rseg, &pcnt = L.vseg;
  rcnt.assign(size_t(L.nr) + 1, 0);
  pcnt.assign(size_t(L.np) + 1, 0);
  {
    // exclusive prefix sums of the counts in (body, thread) order, rigid
    // bodies and particles each from zero (particle entries are numbered
    // after the rigid ones): per chunk of bodies a sum, the chunk starts in
    // order, then each chunk's offsets -- the result of one sequential pass
    auto scan = [&](int b0, int b1, int *seg) {
      const int nb = b1 - b0, nch = layout_threads((long long)nb * nth);
      std::vector<int> part(size_t(nch) + 1, 0);
      parallel_for_threads(nch, [&](int h) {
        const int c0 = b0 + int((long long)nb * h / nch), c1 = b0 + int((long long)nb * (h + 1) / nch);
        int s = 0;
        for (size_t i = size_t(c0) * nth; i < size_t(c1) * nth; i++) s += cnt[i];
        part[size_t(h) + 1] = s;
      });
      for (int h = 0; h < nch; h++) part[size_t(h) + 1] += part[h];
      parallel_for_threads(nch, [&](int h) {
        const int c0 = b0 + int((long long)nb * h / nch), c1 = b0 + int((long long)nb * (h + 1) / nch);
        int run = part[h];
        for (int b = c0; b < c1; b++) {
          for (int k = 0; k < nth; k++) {
            int &x = cnt[size_t(b) * nth + k];
            const int n = x;
            x = run;
            run += n;
          }
          seg[b - b0 + 1] = run;
        }
      });
    };
    scan(0, L.nr, rcnt.data());
    scan(L.nr, nbod, pcnt.data());
  }
  L.ER = rcnt[L.nr];
  L.EV = pcnt[L.np];
  L.eslot.resize(size_t(L.ER) + L.EV);
  L.re0.assign(L.Rpair, -1);
  L.re1.assign(L.Rpair, -1);
  L.te.assign(size_t(12) * L.nt, -1);
  parallel_for_threads(nth, [&](int k) {
    int *ok = cnt.data() + k;
    const long long u0 = nitems * k / nth, u1 = nitems * (k + 1) / nth;
    for (long long u = u0; u < u1; u++)
      visit(u, [&](int row, int slot, int enc) {
        const int b = bidx(enc);
        const int e = (b >= L.nr ? L.ER : 0) + ok[size_t(b) * nth]++;
        if (row < L.Rpair) {
          (slot == 0 ? L.re0 : L.re1)[row] = e;
          L.eslot[e] = 2 * row + slot;
        } else {
          const int tb = (row - L.Rpair) / 3, kk = (row - L.Rpair) % 3;
          L.te[12 * tb + 4 * kk + slot] = e;
          L.eslot[e] = 2 * L.Rpair + 12 * tb + 4 * kk + slot;
        }
      });
  });
  // per-island ranges (each island's bodies, contacts and joints are
  // contiguous in the internal order) and eligibility for the resident CR
  L.ires.assign(size_t(8) * std::max(L.ni, 1), 0);
  L.isres.assign(std::max(L.ni, 1), 0);
  L.isl_rigid.assign(std::max(L.ni, 1), 0);
  {
    std::vector<int> npar(L.ni, 0), ntet(L.ni, 0);
    // an island's items are one run of equal island ids in each list: the
    // thread whose range holds the run's first item records it
    auto runs = [&](int n, auto &&isl_of, auto &&put) {
      const int nth_r = layout_threads(n);
      parallel_for_threads(nth_r, [&](int h) {
        const int i0 = int((long long)n * h / nth_r), i1 = int((long long)n * (h + 1) / nth_r);
        for (int i = i0; i < i1; i++) {
          const int is = isl_of(i);
          if (i > 0 && isl_of(i - 1) == is) continue;
          int j = i + 1;
          while (j < n && isl_of(j) == is) j++;
          put(is, i, j - i);
        }
      });
    };
    auto first = [&](int slot) {
      return [&L, slot](int is, int f, int cnt_) { L.ires[8 * size_t(is) + slot] = f; L.ires[8 * size_t(is) + slot + 1] = cnt_; };
    };
    runs(L.nc, [&](int ci) { return L.risl[3 * size_t(ci)]; }, first(0));
    runs(L.nj, [&](int j) { return L.risl[3 * size_t(L.nc) + 5 * size_t(j)]; }, first(2));
    runs(L.nr, [&](int b) { return L.bisl_r[b]; }, first(4));
    runs(L.np, [&](int b) { return L.bisl_p[b]; }, [&](int is, int, int cnt_) { npar[is] = cnt_; });
    runs(L.nt, [&](int tt) { return L.risl[size_t(L.Rpair) + 3 * size_t(tt)]; }, [&](int is, int, int cnt_) { ntet[is] = cnt_; });
    // (at most 2048 rows: the reduction task table of a group holds 2 per island + rows / 128)
    const int cap = std::min(c->cfg.res_max_rows > 0 ? c->cfg.res_max_rows : 384, 2048);
    for (int i = 0; i < L.ni; i++) L.isl_rigid[i] = npar[i] == 0 && ntet[i] == 0;
    for (int i = 0; i < L.ni; i++) {
      int *r = &L.ires[8 * size_t(i)];
      if (r[5] > 0) { r[6] = L.rseg[r[4]]; r[7] = L.rseg[r[4] + r[5]] - r[6]; }
      const int rows = 3 * r[1] + 5 * r[3];
      if (!c->cfg.cr_resident || npar[i] || ntet[i] || r[5] == 0 || rows == 0 || rows > cap) {
        if (rows > 0 || ntet[i]) L.n_streamed++;
        continue;
      }
      L.isres[i] = 1;
      L.n_res++;
    }
    // groups: runs of consecutive eligible islands (in the internal order, so
    // a group's contacts, joints, bodies and entries are contiguous), at most
    // RES_MAXI islands and `cap` rows each
    L.grp_of.assign(std::max(L.ni, 1), -1);
    std::vector<int> cur;
    int cur_rows = 0;
    auto close = [&]() {
      if (cur.empty()) return;
      const int g = int(L.gres.size() / 10);
      int c0 = -1, nc = 0, j0 = -1, nj = 0, nbg = 0, ent = 0;
      const int b0 = L.ires[8 * size_t(cur[0]) + 4];
      for (int i : cur) {
        const int *r = &L.ires[8 * size_t(i)];
        if (r[1] > 0 && c0 < 0) c0 = r[0];
        if (r[3] > 0 && j0 < 0) j0 = r[2];
        nc += r[1]; nj += r[3]; nbg += r[5]; ent += r[7];
        L.grp_of[i] = g;
      }
      const int e0 = L.rseg[b0];
      const int rec[10] = {std::max(c0, 0), nc, std::max(j0, 0), nj, b0, nbg, e0, ent, int(L.gisl.size()), int(cur.size())};
      L.gres.insert(L.gres.end(), rec, rec + 10);
      L.gisl.insert(L.gisl.end(), cur.begin(), cur.end());
      L.res_rows = std::max(L.res_rows, 3 * nc + 5 * nj);
      L.res_ent = std::max(L.res_ent, ent);
      L.res_bod = std::max(L.res_bod, nbg);
      cur.clear();
      cur_rows = 0;
    };
    for (int i : L.isl_order) {
      if (!L.isres[i]) { close(); continue; }
      const int rows = 3 * L.ires[8 * size_t(i) + 1] + 5 * L.ires[8 * size_t(i) + 3];
      if (int(cur.size()) == RES_MAXI || cur_rows + rows > cap) close();
      cur.push_back(i);
      cur_rows += rows;
    }
    close();
  }
  return NSN_OK;
}

template <typename T>
void carve(Arena &A, Dev<T> &D, const Layout &L, int nb) {
  auto tk = [&](int n) { return A.take<T>(n); };
  for (int k = 0; k < 3; k++) { D.rx[k] = tk(L.nr); D.rx0[k] = tk(L.nr); D.rIb[k] = tk(L.nr); }
  for (int k = 0; k < 4; k++) { D.rq[k] = tk(L.nr); D.rq0[k] = tk(L.nr); }
  for (int k = 0; k < 6; k++) {
    D.ru[k] = tk(L.nr); D.rut[k] = tk(L.nr); D.rIw[k] = tk(L.nr); D.rIwi[k] = tk(L.nr);
    D.rg[k] = tk(L.nr); D.ryg[k] = tk(L.nr);
  }
  D.rm = tk(L.nr); D.rinvm = tk(L.nr);
  for (int k = 0; k < 3; k++) {
    D.px[k] = tk(L.np); D.px0[k] = tk(L.np); D.pu[k] = tk(L.np); D.put[k] = tk(L.np);
    D.phinv[k] = tk(L.np); D.pg[k] = tk(L.np); D.pyg[k] = tk(L.np); D.puprev[k] = tk(L.np);
  }
  D.pm = tk(L.np);
  D.eslot = A.take<int>(size_t(L.ER) + L.EV);
  D.rseg = A.take<int>(L.nr + 1);
  D.vseg = A.take<int>(L.np + 1);
  D.ejA = A.take<RV4<T>>(L.ER);
  D.ejB = A.take<RV2<T>>(L.ER);
  for (int b = 0; b < 2; b++)
    for (int k = 0; k < 3; k++) D.ej3[b][k] = tk(L.EV);
  D.t = tk(2 * L.Rpair + 12 * L.nt);
  D.t2 = tk(2 * L.Rpair + 12 * L.nt);
  D.re0 = A.take<int>(L.Rpair);
  D.re1 = A.take<int>(L.Rpair);
  D.te = A.take<int>(size_t(12) * L.nt);
  D.lam = tk(L.R); D.cdiag = tk(L.R); D.hv = tk(L.R); D.b = tk(L.R); D.P = tk(L.R);
  D.x = tk(L.R); D.z = tk(L.R); D.p = tk(L.R); D.Ap = tk(L.R); D.Az = tk(L.R);
  D.c3 = tk(6 * L.nt);
  D.lam_prev = tk(L.R);
  D.cba = A.take<int>(L.nc); D.cbb = A.take<int>(L.nc);
  for (int k = 0; k < 3; k++) { D.cpa[k] = tk(L.nc); D.cpb[k] = tk(L.nc); D.cn[k] = tk(L.nc); }
  D.cdd = tk(L.nc); D.cmu = tk(L.nc);
  D.cr0 = A.take<double>(sizeof(T) == 4 ? 6 * size_t(L.nc) : 1);
  D.jba = A.take<int>(L.nj); D.jbb = A.take<int>(L.nj);
  for (int k = 0; k < 3; k++) { D.jpa[k] = tk(L.nj); D.jpb[k] = tk(L.nj); D.jaxa[k] = tk(L.nj); D.jaxb[k] = tk(L.nj); }
  D.je = tk(L.nj);
  D.jr0 = A.take<double>(sizeof(T) == 4 ? 15 * size_t(L.nj) : 1);
  D.tv = A.take<int>(4 * L.nt);
  D.tkind = A.take<int>(L.nt);
  D.jkind = A.take<int>(L.nj);
  D.tDmi = tk(9 * L.nt); D.tVe = tk(L.nt); D.tC1 = tk(L.nt); D.tD1 = tk(L.nt); D.talpha = tk(L.nt);
  D.max_blk = device_max_blocks();
  D.part_body = A.take<typename RedT<T>::type>(2 * size_t(D.max_blk));
  D.part_row = A.take<typename RedT<T>::type>(2 * size_t(D.max_blk) * NPART);
  D.sc = A.take<Scalars>(1);
  D.fl = A.take<Flags>(1);
  D.risl = A.take<int>(L.R);
  D.cabi = A.take<int>(L.nc);
  D.row_abi_dev = A.take<int>(L.R);
  D.bisl_r = A.take<int>(L.nr);
  D.bisl_p = A.take<int>(L.np);
  const int ni = std::max(L.ni, 1);
  D.isl.acc = A.take<double>(size_t(ISL_ACC) * ni);
  D.isl.m0 = A.take<double>(ni); D.isl.mf = A.take<double>(ni); D.isl.mw = A.take<double>(ni);
  D.isl.mw2 = A.take<double>(ni);
  D.isl.eta = A.take<double>(ni); D.isl.res0 = A.take<double>(ni); D.isl.rho = A.take<double>(2 * size_t(ni));
  D.isl.res_prev = A.take<double>(ni);
  D.isl.alpha = A.take<double>(ni); D.isl.beta = A.take<double>(ni);
  D.isl.alpha_f = A.take<float>(ni); D.isl.beta_f = A.take<float>(ni);
  D.isl.stop = A.take<int>(ni); D.isl.crdone = A.take<int>(ni);
  D.isl.tacc = A.take<double>(ni);
  D.isl.ls_pre = A.take<int>(ni);
  D.isl.mls = A.take<double>(ni);
  D.isl.rigid = A.take<unsigned char>(ni);
  D.isl.crk = A.take<int>(ni);
  D.isl.mbest = A.take<double>(ni);
  D.isl.bmark = A.take<int>(ni);
  for (int k = 0; k < 6; k++) D.rub[k] = tk(L.nr);
  for (int k = 0; k < 3; k++) D.pub[k] = tk(L.np);
  D.lbest = tk(L.R);
  // line search: du, u and lambda at the head of the Newton iteration, dlambda
  for (int k = 0; k < 6; k++) { D.rdu[k] = tk(L.nr); D.ru0[k] = tk(L.nr); }
  for (int k = 0; k < 3; k++) { D.pdu[k] = tk(L.np); D.pu0[k] = tk(L.np); }
  D.lam0 = tk(L.R); D.xs = tk(L.R);
  D.pscale = tk(std::max(L.nc, 1));
  D.fl_row = A.take<unsigned char>(size_t(L.R) / BLOCK + 1);
  D.fl_br = A.take<unsigned char>(size_t(L.nr) / (BLOCK / 16) + 1);
  D.fl_bp = A.take<unsigned char>(size_t(L.np) / (BLOCK / 16) + 1);
  D.list_row = A.take<int>(size_t(L.R) / BLOCK + 1);
  D.list_br = A.take<int>(size_t(L.nr) / (BLOCK / 16) + 1);
  D.list_bp = A.take<int>(size_t(L.np) / (BLOCK / 16) + 1);
  D.list_isl = A.take<int>(ni);
  D.ires = A.take<int>(size_t(8) * ni);
  D.isres = A.take<unsigned char>(ni);
  const size_t ng = std::max<size_t>(L.gres.size() / 10, 1);
  D.gres = A.take<int>(10 * ng);
  D.gisl = A.take<int>(std::max<size_t>(L.gisl.size(), 1));
  D.grp_of = A.take<int>(ni);
  D.resact = A.take<unsigned char>(ni);
  D.gact = A.take<unsigned char>(ng);
  (void)nb;
}

template <typename T>
void fill_sizes(Dev<T> &D, const Layout &L, const nsn_config &cfg) {
  D.max_blk = device_max_blocks();
  D.nr = L.nr; D.np = L.np; D.nc = L.nc; D.nj = L.nj; D.nt = L.nt; D.R = L.R; D.Rpair = L.Rpair;
  D.ER = L.ER; D.EV = L.EV;
  D.h = cfg.h; D.eps = cfg.eps; D.damping = cfg.damping; D.tol_rel = cfg.tol_rel;
  for (int k = 0; k < 3; k++) D.grav[k] = cfg.gravity[k];
  D.hT = T(cfg.h); D.ihT = T(1.0 / cfg.h); D.epsT = T(cfg.eps); D.dampT = T(cfg.damping);
  for (int k = 0; k < 3; k++) D.gravT[k] = T(cfg.gravity[k]);
  D.ncp = cfg.ncp; D.rscale = cfg.rscale; D.gs = cfg.geom_stiffness; D.cr_tol = cfg.cr_tol_mode;
  D.warm = 0;
  D.ni = L.ni;
  D.isl_on = cfg.island_stop ? 1 : 0;
  D.cone = cfg.cone_project ? 1 : 0;
  D.ls = cfg.line_search ? 1 : 0;
  D.best = cfg.best_iterate && cfg.island_stop ? 1 : 0;
  D.crM = cfg.cr_iters;
  // grid-stride kernels get at most one wave: SMs x resident blocks per SM of
  // the kernel (so that no partial second wave trails the first)
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  auto wave = [&](const void *kern) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, 0) != cudaSuccess || per_sm < 1) per_sm = 8;
    return (long long)nsm * per_sm;
  };
  if (D.G != 4 && D.G != 16) D.G = 8;
  const long long cap_body =
      D.G == 4 ? wave(reinterpret_cast<const void *>(&k_body_pass<T, 4, BM_APPLY>))
               : (D.G == 16 ? wave(reinterpret_cast<const void *>(&k_body_pass<T, 16, BM_APPLY>))
                            : wave(reinterpret_cast<const void *>(&k_body_pass<T, 8, BM_APPLY>)));
  const long long cap_row = cfg.island_stop ? wave(reinterpret_cast<const void *>(&k_row_pass_isl<T, RM_APPLY>))
                                            : wave(reinterpret_cast<const void *>(&k_row_pass<T, RM_APPLY>));
  auto capped = [&](long long n, long long cap) { return int(std::max(1LL, std::min({n, cap, (long long)D.max_blk}))); };
  D.nblk_body_r = L.nr ? capped(cdiv((long long)L.nr * D.G, BLOCK), cap_body) : 0;
  D.nblk_body_p = L.np ? capped(cdiv((long long)L.np * D.G, BLOCK), cap_body) : 0;
  D.nblk_row_pair = L.Rpair ? capped(cdiv(L.Rpair, BLOCK), cap_row) : 0;
  D.nblk_row_tet = L.nt ? capped(cdiv(L.nt, BLOCK), cap_row) : 0;
  D.nblk_upd = clampb(cdiv(std::max(L.R, 1), BLOCK), D.max_blk);
  // island-resident CR: a persistent grid of as many CTAs as fit (shared
  // memory sized for the largest resident island), at most one per island
  D.res_on = 0;
  D.nblk_res = 0;
  D.res_smem = 0;
  D.ngroups = int(L.gres.size() / 10);
  D.streamed = 1;
  if (cfg.island_stop && L.n_res > 0 && D.ngroups > 0) {
    D.res_rows = L.res_rows; D.res_ent = L.res_ent; D.res_bod = L.res_bod;
    const size_t smem = res_smem_bytes<T>(L.res_rows, L.res_ent, L.res_bod);
    int per_sm = 0;
    const void *kern = reinterpret_cast<const void *>(&k_cr_resident<T>);
    // all of the SM's unified L1 / shared memory as shared memory: the
    // resident groups are bound by it (the kernel reads no global data in its loop)
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, int(cudaSharedmemCarveoutMaxShared));
    if (smem <= 200 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RES_THREADS, smem) == cudaSuccess && per_sm > 0) {
      D.res_on = 1;
      D.res_smem = int(smem);
      D.nblk_res = int(std::min<long long>((long long)nsm * per_sm, D.ngroups));
      D.streamed = L.n_streamed > 0 ? 1 : 0;   // 0: no island needs the streamed CR loop
    }
    cudaGetLastError();
  }
}

// host-side copies of per-row / per-body static data, converted to T
template <typename T>
nsn_status upload(nsn_ctx *c, Dev<T> &D) {
  const Layout &L = c->L;
  const HostScene &S = c->scene;
  cudaStream_t st = c->stream;
  // per-field host arrays are written into the pinned stage and copied from there
  PinnedStage &P = c->stage;
  P.rewind();
  bool oom = false;
  auto stage = [&](size_t n) {
    T *q = P.take<T>(n);
    if (!q) oom = true;
    return q;
  };
  auto stagei = [&](size_t n) {
    int *q = P.take<int>(n);
    if (!q) oom = true;
    return q;
  };
  auto put = [&](T *dst, const T *src, size_t n) -> cudaError_t {
    if (!n) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, st);
  };
  auto puti = [&](int *dst, const int *src, size_t n) -> cudaError_t {
    if (!n) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, n * sizeof(int), cudaMemcpyHostToDevice, st);
  };
  auto putv = [&](int *dst, const std::vector<int> &v) { return puti(dst, v.data(), v.size()); };
  const size_t nr = L.nr, np = L.np, nc = L.nc, nj = L.nj, nt = L.nt;
  // rigid static data
  {
    T *m = stage(nr), *im = stage(nr), *I0 = stage(nr), *I1 = stage(nr), *I2 = stage(nr), *pm = stage(np);
    if (oom) return fail(c, NSN_ERR_OUT_OF_MEMORY, "pinned staging of the upload");
    T *I[3] = {I0, I1, I2};
    for (size_t i = 0; i < nr; i++) {
      const int id = L.rig_of[i];
      m[i] = T(S.mass[id]);
      im[i] = T(1.0 / double(S.mass[id]));
      for (int k = 0; k < 3; k++) I[k][i] = T(S.inertia[3 * size_t(id) + k]);
    }
    CUDA_TRY(c, put(D.rm, m, nr)); CUDA_TRY(c, put(D.rinvm, im, nr));
    for (int k = 0; k < 3; k++) CUDA_TRY(c, put(D.rIb[k], I[k], nr));
    for (size_t i = 0; i < np; i++) pm[i] = T(S.mass[L.par_of[i]]);
    CUDA_TRY(c, put(D.pm, pm, np));
  }
  CUDA_TRY(c, putv(D.eslot, L.eslot));
  // slots of world sides are never written and must read as zero
  CUDA_TRY(c, cudaMemsetAsync(D.t, 0, sizeof(T) * std::max(2 * L.Rpair + 12 * L.nt, 1), st));
  CUDA_TRY(c, cudaMemsetAsync(D.t2, 0, sizeof(T) * std::max(2 * L.Rpair + 12 * L.nt, 1), st));
  CUDA_TRY(c, putv(D.rseg, L.rseg));
  CUDA_TRY(c, putv(D.vseg, L.vseg));
  CUDA_TRY(c, putv(D.re0, L.re0));
  CUDA_TRY(c, putv(D.re1, L.re1));
  CUDA_TRY(c, putv(D.te, L.te));
  // contacts
  {
    int *a = stagei(nc), *b = stagei(nc);
    T *f[11];
    for (int k = 0; k < 11; k++) f[k] = stage(nc);
    if (oom) return fail(c, NSN_ERR_OUT_OF_MEMORY, "pinned staging of the upload");
    const int nth = layout_threads((long long)nc);
    parallel_for_threads(nth, [&](int k0) {
      const size_t i0 = nc * size_t(k0) / nth, i1 = nc * size_t(k0 + 1) / nth;
      for (size_t i = i0; i < i1; i++) {
        const nsn_contact &r = S.contacts[L.cperm[i]];
        a[i] = r.body_a >= 0 ? L.bmap[r.body_a] : -1;
        b[i] = r.body_b >= 0 ? L.bmap[r.body_b] : -1;
        for (int k = 0; k < 3; k++) { f[k][i] = T(r.pa[k]); f[3 + k][i] = T(r.pb[k]); f[6 + k][i] = T(r.n[k]); }
        f[9][i] = T(r.d); f[10][i] = T(r.mu);
      }
    });
    CUDA_TRY(c, puti(D.cba, a, nc)); CUDA_TRY(c, puti(D.cbb, b, nc));
    for (int k = 0; k < 3; k++) {
      CUDA_TRY(c, put(D.cpa[k], f[k], nc)); CUDA_TRY(c, put(D.cpb[k], f[3 + k], nc)); CUDA_TRY(c, put(D.cn[k], f[6 + k], nc));
    }
    CUDA_TRY(c, put(D.cdd, f[9], nc)); CUDA_TRY(c, put(D.cmu, f[10], nc));
  }
  // joints
  {
    int *a = stagei(nj), *b = stagei(nj), *jk = stagei(nj);
    T *f[13];
    for (int k = 0; k < 13; k++) f[k] = stage(nj);
    if (oom) return fail(c, NSN_ERR_OUT_OF_MEMORY, "pinned staging of the upload");
    for (size_t i = 0; i < nj; i++) {
      const nsn_revolute &r = S.joints[L.jperm[i]];
      a[i] = r.body_a >= 0 ? L.bmap[r.body_a] : -1;
      b[i] = r.body_b >= 0 ? L.bmap[r.body_b] : -1;
      for (int k = 0; k < 3; k++) {
        f[k][i] = T(r.pa[k]); f[3 + k][i] = T(r.pb[k]); f[6 + k][i] = T(r.axis_a[k]); f[9 + k][i] = T(r.axis_b[k]);
      }
      f[12][i] = T(r.compliance);
      jk[i] = S.jkind[L.jperm[i]];
    }
    CUDA_TRY(c, puti(D.jba, a, nj)); CUDA_TRY(c, puti(D.jbb, b, nj));
    for (int k = 0; k < 3; k++) {
      CUDA_TRY(c, put(D.jpa[k], f[k], nj)); CUDA_TRY(c, put(D.jpb[k], f[3 + k], nj));
      CUDA_TRY(c, put(D.jaxa[k], f[6 + k], nj)); CUDA_TRY(c, put(D.jaxb[k], f[9 + k], nj));
    }
    CUDA_TRY(c, put(D.je, f[12], nj));
    CUDA_TRY(c, puti(D.jkind, jk, nj));
  }
  // tets: rest-shape inverse, volume and stable Neo-Hookean constants (App. B):
  // C1 = mu/2, D1 = lambda/2 (Lame), alpha = 1 + mu/lambda (rest state stress
  // free).  A block of a linear tet (Sec. 9.2.1) holds, in place of (C1, D1,
  // alpha), the compliances E' = 1 / (V_e k) of its three modes: the isotropic
  // stiffness of the engineering strains has the eigenvalue 3 lambda + 2 mu on
  // the volumetric mode, 2 mu on the two deviatoric normal modes and mu on the
  // three shears, so (V_e K_e)^-1 is diagonal in that basis.
  {
    int *v = stagei(4 * nt), *kind = stagei(nt);
    T *Dmi = stage(9 * nt), *Ve = stage(nt), *C1 = stage(nt), *D1 = stage(nt), *al = stage(nt);
    if (oom) return fail(c, NSN_ERR_OUT_OF_MEMORY, "pinned staging of the upload");
    for (size_t t = 0; t < nt; t++) {
      const nsn_tet &r = *L.tb_rec[L.tperm[t]];
      kind[t] = L.tb_kind[L.tperm[t]];
      for (int q = 0; q < 4; q++) v[4 * t + q] = -L.bmap[r.v[q]] - 2;
      double Dm[9];
      for (int row = 0; row < 3; row++)
        for (int k = 0; k < 3; k++) Dm[3 * row + k] = double(r.rest[k + 1][row]) - double(r.rest[0][row]);
      double det = Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
                   Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
      double inv[9] = {(Dm[4] * Dm[8] - Dm[5] * Dm[7]) / det, (Dm[2] * Dm[7] - Dm[1] * Dm[8]) / det,
                       (Dm[1] * Dm[5] - Dm[2] * Dm[4]) / det, (Dm[5] * Dm[6] - Dm[3] * Dm[8]) / det,
                       (Dm[0] * Dm[8] - Dm[2] * Dm[6]) / det, (Dm[2] * Dm[3] - Dm[0] * Dm[5]) / det,
                       (Dm[3] * Dm[7] - Dm[4] * Dm[6]) / det, (Dm[1] * Dm[6] - Dm[0] * Dm[7]) / det,
                       (Dm[0] * Dm[4] - Dm[1] * Dm[3]) / det};
      for (int k = 0; k < 9; k++) Dmi[9 * t + k] = T(inv[k]);
      Ve[t] = T(std::fabs(det) / 6.0);
      double mu = double(r.E) / (2.0 * (1.0 + double(r.nu)));
      double la = double(r.E) * double(r.nu) / ((1.0 + double(r.nu)) * (1.0 - 2.0 * double(r.nu)));
      const double V = std::fabs(det) / 6.0;
      if (kind[t] == 0) {
        C1[t] = T(0.5 * mu); D1[t] = T(0.5 * la); al[t] = T(1.0 + mu / la);
      } else if (kind[t] == 1) {
        C1[t] = T(1.0 / (V * (3.0 * la + 2.0 * mu))); D1[t] = T(1.0 / (V * 2.0 * mu)); al[t] = D1[t];
      } else {
        C1[t] = T(1.0 / (V * mu)); D1[t] = C1[t]; al[t] = C1[t];
      }
    }
    CUDA_TRY(c, puti(D.tv, v, 4 * nt));
    CUDA_TRY(c, puti(D.tkind, kind, nt));
    CUDA_TRY(c, put(D.tDmi, Dmi, 9 * nt)); CUDA_TRY(c, put(D.tVe, Ve, nt)); CUDA_TRY(c, put(D.tC1, C1, nt));
    CUDA_TRY(c, put(D.tD1, D1, nt)); CUDA_TRY(c, put(D.talpha, al, nt));
  }
  {
    T *ones = stage(std::max<size_t>(nc, 1));
    if (oom) return fail(c, NSN_ERR_OUT_OF_MEMORY, "pinned staging of the upload");
    for (size_t i = 0; i < std::max<size_t>(nc, 1); i++) ones[i] = T(1);
    CUDA_TRY(c, put(D.pscale, ones, std::max<size_t>(nc, 1)));
  }
  CUDA_TRY(c, cudaMemsetAsync(D.lam, 0, sizeof(T) * std::max(L.R, 1), st));
  CUDA_TRY(c, cudaMemsetAsync(D.lam_prev, 0, sizeof(T) * std::max(L.R, 1), st));
  CUDA_TRY(c, cudaMemsetAsync(D.sc, 0, sizeof(Scalars), st));
  CUDA_TRY(c, cudaMemsetAsync(D.fl, 0, sizeof(Flags), st));
  CUDA_TRY(c, putv(D.risl, L.risl));
  CUDA_TRY(c, putv(D.cabi, L.cperm));
  CUDA_TRY(c, putv(D.row_abi_dev, L.row_abi));
  CUDA_TRY(c, putv(D.bisl_r, L.bisl_r));
  CUDA_TRY(c, putv(D.bisl_p, L.bisl_p));
  CUDA_TRY(c, putv(D.ires, L.ires));
  CUDA_TRY(c, cudaMemcpyAsync(D.isres, L.isres.data(), L.isres.size(), cudaMemcpyHostToDevice, st));
  CUDA_TRY(c, cudaMemcpyAsync(D.isl.rigid, L.isl_rigid.data(), L.isl_rigid.size(), cudaMemcpyHostToDevice, st));
  CUDA_TRY(c, cudaMemsetAsync(D.isl.ls_pre, 0, sizeof(int) * size_t(std::max(L.ni, 1)), st));
  CUDA_TRY(c, putv(D.gres, L.gres));
  CUDA_TRY(c, putv(D.gisl, L.gisl));
  CUDA_TRY(c, putv(D.grp_of, L.grp_of));
  CUDA_TRY(c, cudaMemsetAsync(D.resact, 0, size_t(std::max(L.ni, 1)), st));
  CUDA_TRY(c, cudaMemsetAsync(D.gact, 0, std::max<size_t>(L.gres.size() / 10, 1), st));
  {
    const size_t ni = size_t(std::max(L.ni, 1));
    CUDA_TRY(c, cudaMemsetAsync(D.isl.acc, 0, sizeof(double) * ISL_ACC * ni, st));
    CUDA_TRY(c, cudaMemsetAsync(D.isl.m0, 0, sizeof(double) * ni, st));
    CUDA_TRY(c, cudaMemsetAsync(D.isl.mf, 0, sizeof(double) * ni, st));
    CUDA_TRY(c, cudaMemsetAsync(D.isl.mw, 0, sizeof(double) * ni, st));
    CUDA_TRY(c, cudaMemsetAsync(D.isl.stop, 0xff, sizeof(int) * ni, st));
    CUDA_TRY(c, cudaMemsetAsync(D.isl.crdone, 0, sizeof(int) * ni, st));
    CUDA_TRY(c, cudaMemsetAsync(D.fl_row, 1, size_t(L.R) / BLOCK + 1, st));
    CUDA_TRY(c, cudaMemsetAsync(D.fl_br, 1, size_t(L.nr) / (BLOCK / 16) + 1, st));
    CUDA_TRY(c, cudaMemsetAsync(D.fl_bp, 1, size_t(L.np) / (BLOCK / 16) + 1, st));
  }
  for (int b2 = 0; b2 < 2; b2++)
    for (int k = 0; k < 3; k++)
      if (L.EV) CUDA_TRY(c, cudaMemsetAsync(D.ej3[b2][k], 0, sizeof(T) * L.EV, st));
  return NSN_OK;
}

// ------------------------------------------------------------------------------------
// state transfer (AoS float <-> SoA T)

template <typename T>
__global__ void k_scatter_state(Dev<T> D, const int *bmap, int nb, const float *pos, const float *quat,
                                const float *vel, const float *omega) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int e = bmap[i];
  if (e >= 0) {
    for (int k = 0; k < 3; k++) {
      if (pos) D.rx[k][e] = T(pos[3 * i + k]);
      if (vel) D.ru[k][e] = T(vel[3 * i + k]);
      if (omega) D.ru[3 + k][e] = T(omega[3 * i + k]);
    }
    if (quat)
      for (int k = 0; k < 4; k++) D.rq[k][e] = T(quat[4 * i + k]);
  } else {
    int p = -e - 2;
    for (int k = 0; k < 3; k++) {
      if (pos) D.px[k][p] = T(pos[3 * i + k]);
      if (vel) D.pu[k][p] = T(vel[3 * i + k]);
    }
  }
}

template <typename T, typename O = float>
__global__ void k_gather_state(Dev<T> D, const int *bmap, int nb, O *pos, O *quat, O *vel,
                               O *omega) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int e = bmap[i];
  if (e >= 0) {
    for (int k = 0; k < 3; k++) {
      if (pos) pos[3 * i + k] = O(D.rx[k][e]);
      if (vel) vel[3 * i + k] = O(D.ru[k][e]);
      if (omega) omega[3 * i + k] = O(D.ru[3 + k][e]);
    }
    if (quat)
      for (int k = 0; k < 4; k++) quat[4 * i + k] = O(D.rq[k][e]);
  } else {
    int p = -e - 2;
    for (int k = 0; k < 3; k++) {
      if (pos) pos[3 * i + k] = O(D.px[k][p]);
      if (vel) vel[3 * i + k] = O(D.pu[k][p]);
      if (omega) omega[3 * i + k] = O(0);
    }
    if (quat) { quat[4 * i] = O(1); quat[4 * i + 1] = quat[4 * i + 2] = quat[4 * i + 3] = O(0); }
  }
}

// copies of the committed state (x, q, u) for nsn_linearize
template <typename T>
__global__ void k_backup_state(Dev<T> D, T *buf, int restore) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nr = D.nr, np = D.np;
  if (i < nr) {
    T *b = buf + 13 * size_t(i);
    for (int k = 0; k < 3; k++) { if (restore) D.rx[k][i] = b[k]; else b[k] = D.rx[k][i]; }
    for (int k = 0; k < 4; k++) { if (restore) D.rq[k][i] = b[3 + k]; else b[3 + k] = D.rq[k][i]; }
    for (int k = 0; k < 6; k++) { if (restore) D.ru[k][i] = b[7 + k]; else b[7 + k] = D.ru[k][i]; }
  } else if (i < nr + np) {
    int p = i - nr;
    T *b = buf + 13 * size_t(i);
    for (int k = 0; k < 3; k++) { if (restore) D.px[k][p] = b[k]; else b[k] = D.px[k][p]; }
    for (int k = 0; k < 3; k++) { if (restore) D.pu[k][p] = b[3 + k]; else b[3 + k] = D.pu[k][p]; }
  }
}

// ------------------------------------------------------------------------------------
// step orchestration

nsn_status mlp_infer(nsn_ctx *c, const float *X, int n, float *Y, cudaStream_t st);
nsn_status mlp_check(nsn_ctx *c, cudaStream_t st);

template <typename T>
struct Launcher {
  nsn_ctx *c;
  Dev<T> &D;
  cudaStream_t st;
  int count = 0;

  void body(int mode, const T *in, int buf, int it, int force) {
    int nb = D.nblk_body_r + D.nblk_body_p;
    if (!nb) return;
    if (D.G == 4) body_g<4>(mode, nb, in, buf, it, force);
    else if (D.G == 16) body_g<16>(mode, nb, in, buf, it, force);
    else body_g<8>(mode, nb, in, buf, it, force);
    count++;
  }
  template <int G>
  void body_g(int mode, int nb, const T *in, int buf, int it, int force) {
    if (mode == BM_RESIDUAL) k_body_pass<T, G, BM_RESIDUAL><<<nb, BLOCK, 0, st>>>(D, in, buf, it, force);
    else if (mode == BM_APPLY) k_body_pass<T, G, BM_APPLY><<<nb, BLOCK, 0, st>>>(D, in, buf, it, force);
    else k_body_pass<T, G, BM_UPDATE><<<nb, BLOCK, 0, st>>>(D, in, buf, it, force);
  }
  void rows(int mode, int force) {
    int nb = D.nblk_row_pair + D.nblk_row_tet;
    if (!nb) return;
    if (D.isl_on) {
      if (mode == RM_RHS) k_row_pass_isl<T, RM_RHS><<<nb, BLOCK, 0, st>>>(D, force);
      else if (mode == RM_MERIT) k_row_pass_isl<T, RM_MERIT><<<nb, BLOCK, 0, st>>>(D, force);
      else k_row_pass_isl<T, RM_APPLY><<<nb, BLOCK, 0, st>>>(D, force);
    } else if (mode == RM_RHS) k_row_pass<T, RM_RHS><<<nb, BLOCK, 0, st>>>(D, force);
    else if (mode == RM_MERIT) k_row_pass<T, RM_MERIT><<<nb, BLOCK, 0, st>>>(D, force);
    else k_row_pass<T, RM_APPLY><<<nb, BLOCK, 0, st>>>(D, force);
    count++;
  }
  // merit of an evaluation (island mode: the per-island pass first); the
  // k_merit launch itself is counted by the callers
  void merit(int n, int force, double trial_t = 0.0) {
    if (D.isl_on) {
      if (!force) {   // a Newton iteration: new work lists
        k_list_reset<T><<<1, 1, 0, st>>>(D);
        count++;
        if (D.res_on) cudaMemsetAsync(D.gact, 0, size_t(D.ngroups), st);
      }
      k_merit_isl<T><<<cdiv(std::max(D.ni, 1), 256), 256, 0, st>>>(D, n, force, trial_t);
      count++;
    }
    k_merit<T><<<1, RED_THREADS, 0, st>>>(D, n, force, trial_t);
  }
  void eval(int buf, int force) {
    if (D.nc) { k_eval_contacts<T><<<cdiv(D.nc, 128), 128, 0, st>>>(D, buf, force); count++; }
    if (D.nj) { k_eval_joints<T><<<cdiv(D.nj, 128), 128, 0, st>>>(D, buf, force); count++; }
    if (D.nt) { k_eval_tets<T><<<cdiv(D.nt, 128), 128, 0, st>>>(D, buf, force); count++; }
  }
  void begin() {
    // plain start of Sec. 8.1: lambda^0 = 0 (u^0 = 0 is set by the begin kernels)
    if (D.R) cudaMemsetAsync(D.lam, 0, sizeof(T) * D.R, st);
    if (D.isl_on && D.ni) {
      if (D.best) {   // least merits start above any finite merit (0x7f bytes: 1.4e306)
        cudaMemsetAsync(D.isl.mbest, 0x7f, sizeof(double) * D.ni, st);
        cudaMemsetAsync(D.isl.bmark, 0, sizeof(int) * D.ni, st);
      }
      cudaMemsetAsync(D.isl.stop, 0xff, sizeof(int) * D.ni, st);
      cudaMemsetAsync(D.isl.acc, 0, sizeof(double) * ISL_ACC * D.ni, st);
      cudaMemsetAsync(D.isl.ls_pre, 0, sizeof(int) * D.ni, st);   // no line-search evaluation carries over
    }
    k_begin_rigid<T><<<cdiv(std::max(D.nr, 1), 128), 128, 0, st>>>(D);
    count++;
    if (D.np) { k_begin_particle<T><<<cdiv(D.np, 128), 128, 0, st>>>(D); count++; }
    if (sizeof(T) == 4 && D.nc) { k_contact_r0<T><<<cdiv(D.nc, 256), 256, 0, st>>>(D); count++; }
    if (sizeof(T) == 4 && D.nj) { k_joint_r0<T><<<cdiv(D.nj, 128), 128, 0, st>>>(D); count++; }
  }
  void linearize_at(int n) {  // rows, g, H~, b, diag at Newton iteration n (or IT_DEV)
    const int buf = n == IT_DEV ? IT_DEV : (n & 1);
    eval(buf, 0);
    body(BM_RESIDUAL, D.lam, buf, n, 0);
    rows(RM_RHS, 0);
    merit(n, 0);
    count++;
  }
  void cr_begin(int M) {
    k_cr_begin<T><<<1, 1, 0, st>>>(D, M);
    count++;
  }
  void cr_body(int buf, int M) {  // one CR iteration (index read on the device)
    body(BM_APPLY, D.z, buf, 0, 0);
    rows(RM_APPLY, 0);
    if (D.isl_on) {
      k_cr_scalars_isl<T><<<cdiv(std::max(D.ni, 1), 256), 256, 0, st>>>(D);
      k_cr_update_isl<T><<<D.nblk_upd, BLOCK, 0, st>>>(D);
    } else {
      k_cr_scalars<T><<<1, RED_THREADS, 0, st>>>(D);
      k_cr_update<T><<<D.nblk_upd, BLOCK, 0, st>>>(D);
    }
    k_cr_next<T><<<1, 1, 0, st>>>(D, M);
    count += 3;
  }
  void cr(int iters, int buf) {  // eager CR loop
    if (!D.R) return;
    cr_begin(iters);
    for (int k = 0; k < iters; k++) cr_body(buf, iters);
  }
  void newton_update(int n) {
    const int buf = n == IT_DEV ? IT_DEV : (n & 1);
    body(BM_UPDATE, D.x, buf, n, 0);
    k_lambda_update<T><<<D.nblk_upd, BLOCK, 0, st>>>(D);
    count++;
  }
  // warm start of Sec. 8.1's multipliers (previous step or learned), kept only
  // if the merit at (u = 0, lambda^0) does not exceed the zero start's
  void warm_start() {
    eval(0, 1);
    body(BM_RESIDUAL, D.lam, 0, 0, 1);
    rows(RM_RHS, 1);
    merit(-1, 1);
    count++;
    // previous-step candidate (also the fallback of the learned start)
    if (D.R) { k_warm_from_prev<T><<<D.nblk_upd, BLOCK, 0, st>>>(D, c->warm_friction); count++; }
    eval(0, 1);
    body(BM_RESIDUAL, D.lam, 0, 0, 1);
    rows(RM_RHS, 1);
    merit(-2, 1);
    count++;
    if (c->warm_mode == NSN_WARM_PREV) {
      k_warm_accept<T><<<D.nblk_upd, BLOCK, 0, st>>>(D);
      count++;
      return;
    }
    // learned candidate: contacts from the network, joint and tet rows zero
    if (D.R) cudaMemsetAsync(D.lam, 0, sizeof(T) * D.R, st);
    if (D.nc) { k_warm_from_pred<T><<<cdiv(D.nc, 128), 128, 0, st>>>(D, c->mlp.Y, c->warm_friction); count++; }
    eval(0, 1);
    body(BM_RESIDUAL, D.lam, 0, 0, 1);
    rows(RM_RHS, 1);
    merit(-4, 1);
    k_warm_choose<T><<<D.nblk_upd, BLOCK, 0, st>>>(D, c->warm_friction);
    count += 2;
  }
  // segments of one step (Algorithm 1): prefix, Newton loop body (head, CR
  // loop body, tail), suffix
  void prefix() {
    if (c->warm_mode == NSN_WARM_LEARNED && D.nc) {
      k_contact_features<T><<<cdiv(D.nc, 128), 128, 0, st>>>(D, c->mlp.X);
      count++;
      mlp_infer(c, c->mlp.X, D.nc, c->mlp.Y, st);
      count++;
    }
    begin();
    if (c->warm_mode != NSN_WARM_ZERO) warm_start();
  }
  void newton_head(int M) {
    linearize_at(IT_DEV);
    if (D.isl_on) {
      const int gb = BLOCK / D.G;
      const int nblk = std::max({cdiv(std::max(D.R, 1), BLOCK), cdiv(D.nr, gb), cdiv(D.np, gb), 1});
      if (D.streamed) {   // work lists of the streamed CR loop
        k_block_flags<T><<<nblk, BLOCK, 0, st>>>(D);
        k_block_lists<T><<<1, 1024, 0, st>>>(D, 0);
        count += 2;
      }
      if (D.res_on && M > 0) {
        k_cr_resident<T><<<D.nblk_res, RES_THREADS, D.res_smem, st>>>(D, M);
        count++;
      }
    }
    if (D.R && M > 0 && D.streamed) cr_begin(M);
  }
  // back-tracking line search on the Newton step (Sec. 8.1): five trials t = 1,
  // 1/2, 1/4, 1/8, 1/16, each a merit evaluation at the trial iterate (rows into
  // the next iteration's entry buffer, no geometric stiffness, |h|^2 only in the
  // row pass), then the accepted step (or the damping) committed
  void line_search() {
    body(BM_UPDATE, D.x, IT_DEV, IT_DEV, 0);   // du and the iterate kept, nothing committed
    const int nl = D.nr + D.np + D.R;
    const int gl = clampb(cdiv(std::max(nl, 1), 256), D.max_blk);
    k_ls_begin<T><<<D.nblk_upd, BLOCK, 0, st>>>(D);
    count++;
    T t = T(1);
    for (int j = 0; j < 5; j++, t *= T(0.5)) {
      k_ls_set<T><<<gl, 256, 0, st>>>(D, t, 0);
      eval(IT_DEV_NEXT, 0);
      body(BM_RESIDUAL, D.lam, IT_DEV_NEXT, 0, 0);
      rows(RM_MERIT, 0);
      merit(IT_TRIAL, 1, double(t));
      count += 2;
    }
    k_ls_set<T><<<gl, 256, 0, st>>>(D, T(0), 1);
    count++;
  }
  void newton_tail(int N) {
    if (D.ls && D.R) line_search();
    else newton_update(IT_DEV);
    k_newton_next<T><<<1, 1, 0, st>>>(D, N);
    count++;
  }
  void suffix() {  // merit at the returned iterate, multipliers kept for warm starts
    eval(IT_DEV, 1);
    body(BM_RESIDUAL, D.lam, IT_DEV, IT_DEV, 1);
    rows(RM_RHS, 1);
    merit(IT_FINAL, 1);
    count++;
    if (D.best && D.ni) {   // islands whose last iterate is not their least-merit one
      const int n = D.nr + D.np + D.R;
      k_best_restore<T><<<clampb(cdiv(std::max(n, 1), 256), D.max_blk), 256, 0, st>>>(D);
      k_best_final<T><<<1, RED_THREADS, 0, st>>>(D);
      count += 2;
    }
    if (D.R) { k_copy<T><<<D.nblk_upd, BLOCK, 0, st>>>(D.lam_prev, D.lam, D.R); count++; }
  }
  void step() {  // eager launch of the whole step
    const int N = c->cfg.newton_iters, M = c->cfg.cr_iters;
    prefix();
    for (int n = 0; n < N; n++) {
      newton_head(M);
      if (D.R && M > 0 && D.streamed)
        for (int k = 0; k < M; k++) cr_body(IT_DEV, M);
      newton_tail(N);
    }
    suffix();
  }
};

// island mode: every block of rows and bodies takes part (verification paths
// that run CR without the per-Newton-iteration block flags)
template <typename T>
void blocks_all_on(Dev<T> &D, cudaStream_t st) {
  if (!D.isl_on) return;
  cudaMemsetAsync(D.fl_row, 1, size_t(D.R) / BLOCK + 1, st);
  cudaMemsetAsync(D.fl_br, 1, size_t(D.nr) / (BLOCK / 16) + 1, st);
  cudaMemsetAsync(D.fl_bp, 1, size_t(D.np) / (BLOCK / 16) + 1, st);
  k_block_lists<T><<<1, 1024, 0, st>>>(D, 1);
}

template <typename T>
Dev<T> &dev(nsn_ctx *c);
template <>
Dev<float> &dev<float>(nsn_ctx *c) { return c->d32; }
template <>
Dev<double> &dev<double>(nsn_ctx *c) { return c->d64; }

nsn_status ensure_built(nsn_ctx *c);

// Autotuner of the body pass's segment tile: on large scenes, time the
// operator's body pass (every body active) with 4, 8 and 16 lanes per body on
// this layout.  8 is kept unless another tile is at least 10% faster: the tile
// also sets the granularity of the skip blocks of bodies (BLOCK / G), and late
// in a step, when few islands still iterate, 8 lanes (32-body blocks) skip
// finer than 4 (64-body blocks).  Small scenes take 8 (launch-bound).
template <typename T>
nsn_status tune_body(nsn_ctx *c, Dev<T> &D) {
  const Layout &L = c->L;
  cudaStream_t st = c->stream;
  if (!c->forced_lanes && c->tuned_lanes && c->tuned_nb == L.nr + L.np && L.R >= 100000) {
    // rebuilt for new contacts: same bodies, same tile (and the times measured for it)
    D.G = c->tuned_lanes;
    fill_sizes(D, L, c->cfg);
    return NSN_OK;
  }
  c->tune_ms[0] = c->tune_ms[1] = c->tune_ms[2] = 0.f;
  if (c->forced_lanes) {
    D.G = c->forced_lanes;
    fill_sizes(D, L, c->cfg);
    return NSN_OK;
  }
  if (L.R < 100000 || (L.nr + L.np) == 0) {
    D.G = 8;
    fill_sizes(D, L, c->cfg);
    return NSN_OK;
  }
  if (L.R) CUDA_TRY(c, cudaMemsetAsync(D.z, 0, sizeof(T) * L.R, st));
  cudaEvent_t e0, e1;
  CUDA_TRY(c, cudaEventCreate(&e0));
  CUDA_TRY(c, cudaEventCreate(&e1));
  const int cand[3] = {4, 8, 16};
  int best = 8;
  float best_ms = 1e30f;
  for (int k = 0; k < 3; k++) {
    D.G = cand[k];
    fill_sizes(D, L, c->cfg);
    Launcher<T> Lr{c, D, st};
    Lr.body(BM_APPLY, D.z, 0, 0, 1);  // warm-up
    CUDA_TRY(c, cudaEventRecord(e0, st));
    for (int r = 0; r < 3; r++) Lr.body(BM_APPLY, D.z, 0, 0, 1);
    CUDA_TRY(c, cudaEventRecord(e1, st));
    CUDA_TRY(c, cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    c->tune_ms[k] = ms / 3;
  }
  best_ms = c->tune_ms[1];
  for (int k : {0, 2})
    if (c->tune_ms[k] < 0.9f * best_ms) { best_ms = c->tune_ms[k]; best = cand[k]; }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  D.G = best;
  c->tuned_lanes = best;
  c->tuned_nb = L.nr + L.np;
  fill_sizes(D, L, c->cfg);
  CUDA_TRY(c, cudaGetLastError());
  return NSN_OK;
}

template <typename T>
nsn_status build_device(nsn_ctx *c) {
  const Layout &L = c->L;
  const int nb = int(c->scene.kind.size());
  Dev<T> &D = dev<T>(c);
  D = Dev<T>();
  fill_sizes(D, L, c->cfg);
  Arena A;
  carve(A, D, L, nb);
  size_t need = A.off + size_t(256) * 4 + sizeof(int) * nb + sizeof(float) * 13 * (nb + 1) + sizeof(T) * 13 * (nb + 1);
  // a rebuild (contacts regenerated) reuses the allocation when it still fits;
  // a new one has 25% of headroom for the next contact sets
  if (!c->dmem || need > c->dcap) {
    if (c->dmem) { cudaFree(c->dmem); c->dmem = nullptr; c->dcap = 0; }
    const size_t cap = need + need / 4;
    cudaError_t e = cudaMalloc(&c->dmem, cap);
    if (e != cudaSuccess) return fail(c, NSN_ERR_OUT_OF_MEMORY, "cudaMalloc(%zu): %s", cap, cudaGetErrorString(e));
    c->dcap = cap;
  }
  c->dbytes = need;
  A.base = static_cast<char *>(c->dmem);
  A.sizing = false;
  A.off = 0;
  carve(A, D, L, nb);
  fill_sizes(D, L, c->cfg);
  c->d_bmap = A.take<int>(nb);
  c->d_stage = A.take<float>(13 * size_t(nb + 1));
  c->d_backup = reinterpret_cast<float *>(A.take<T>(13 * size_t(nb + 1)));
  nsn_status s = upload<T>(c, D);
  if (s != NSN_OK) return s;
  if ((s = tune_body<T>(c, D)) != NSN_OK) return s;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_bmap, L.bmap.data(), sizeof(int) * std::max(nb, 0), cudaMemcpyHostToDevice, c->stream));
  // initial state
  const HostScene &S = c->scene;
  float *st = c->d_stage;
  float *dpos = st, *dquat = st + 3 * nb, *dvel = st + 7 * nb, *dom = st + 10 * nb;
  if (nb && c->keep_state_ready && c->keep_state_n >= 13 * size_t(nb)) {
    // a rebuild with the same bodies: the state kept on the device (same layout)
    CUDA_TRY(c, cudaMemcpyAsync(st, c->keep_state, sizeof(float) * 13 * size_t(nb), cudaMemcpyDeviceToDevice, c->stream));
    k_scatter_state<T><<<cdiv(nb, 128), 128, 0, c->stream>>>(D, c->d_bmap, nb, dpos, dquat, dvel, dom);
    CUDA_TRY(c, cudaGetLastError());
  } else if (nb) {
    CUDA_TRY(c, cudaMemcpyAsync(dpos, S.pos.data(), sizeof(float) * 3 * nb, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(dquat, S.quat.data(), sizeof(float) * 4 * nb, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(dvel, S.vel.data(), sizeof(float) * 3 * nb, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(dom, S.omega.data(), sizeof(float) * 3 * nb, cudaMemcpyHostToDevice, c->stream));
    k_scatter_state<T><<<cdiv(nb, 128), 128, 0, c->stream>>>(D, c->d_bmap, nb, dpos, dquat, dvel, dom);
    CUDA_TRY(c, cudaGetLastError());
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return NSN_OK;
}

}  // namespace
nsn_status state_io(nsn_ctx *c, bool set, bool device, const float *ipos, const float *iquat,
                    const float *ivel, const float *iom, float *opos, float *oquat, float *ovel, float *oom);
namespace {

// Key of a contact for matching across regenerations: its two bodies and the
// bit patterns of its body-local point on a (for a generated contact, the
// vertex: a box corner, or the particle).
// The previous step's multipliers of the built scene, in ABI row order
// (empty if there is no built scene), to carry over a rebuild.
template <typename T>
nsn_status save_lam_prev(nsn_ctx *c, std::vector<double> &out) {
  out.clear();
  const Dev<T> &D = dev<T>(c);
  const Layout &L = c->L;
  if (!c->dmem || L.R == 0 || !D.lam_prev) return NSN_OK;
  c->stage.rewind();
  T *v = c->stage.take<T>(L.R);
  if (!v) return fail(c, NSN_ERR_OUT_OF_MEMORY, "pinned staging of the previous multipliers");
  CUDA_TRY(c, cudaMemcpyAsync(v, D.lam_prev, sizeof(T) * L.R, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  out.resize(L.R);
  for (int i = 0; i < L.R; i++) out[L.row_abi[i]] = double(v[i]);
  return NSN_OK;
}

// lam_prev of the new build: row i takes the kept multiplier of the old
// internal row that the map assigns to its ABI row (-1: zero)
template <typename T>
__global__ void k_gather_lam(T *dst, const T *src, const int *map_abi, const int *row_abi, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int o = map_abi[row_abi[i]];
    dst[i] = o >= 0 ? src[o] : T(0);
  }
}

// Before a rebuild (contacts replaced, the layout built anew): the device's
// state, in ABI order, and its previous-step multipliers, in the old internal
// row order, are copied aside on the device, with the old internal index of
// every ABI contact, joint and tet block (host), so that the new build takes
// them over without a round trip through the host.
template <typename T>
nsn_status keep_for_rebuild(nsn_ctx *c) {
  const Dev<T> &D = dev<T>(c);
  const Layout &L = c->L;
  const size_t nb = size_t(c->built_nb);
  if (c->keep_state_n < 13 * nb) {
    if (c->keep_state) cudaFree(c->keep_state);
    c->keep_state = nullptr;
    c->keep_state_n = 0;
    CUDA_TRY(c, cudaMalloc(&c->keep_state, sizeof(float) * 13 * nb));
    c->keep_state_n = 13 * nb;
  }
  float *p = c->keep_state;
  c->dirty = false;
  nsn_status s = state_io(c, false, true, nullptr, nullptr, nullptr, nullptr, p, p + 3 * nb, p + 7 * nb, p + 10 * nb);
  c->dirty = true;
  if (s != NSN_OK) return s;
  const size_t bytes = sizeof(T) * std::max(L.R, 1);
  if (c->keep_lam_bytes < bytes) {
    if (c->keep_lam) cudaFree(c->keep_lam);
    c->keep_lam = nullptr;
    c->keep_lam_bytes = 0;
    CUDA_TRY(c, cudaMalloc(&c->keep_lam, bytes));
    c->keep_lam_bytes = bytes;
  }
  if (L.R) CUDA_TRY(c, cudaMemcpyAsync(c->keep_lam, D.lam_prev, sizeof(T) * L.R, cudaMemcpyDeviceToDevice, c->stream));
  c->old_cinv.resize(L.nc);
  for (int ci = 0; ci < L.nc; ci++) c->old_cinv[L.cperm[ci]] = ci;
  c->old_jinv.resize(L.nj);
  for (int j = 0; j < L.nj; j++) c->old_jinv[L.jperm[j]] = j;
  c->old_tinv.resize(L.nt);
  for (int tb = 0; tb < L.nt; tb++) c->old_tinv[L.tperm[tb]] = tb;
  c->old_nc = L.nc;
  c->old_Rpair = L.Rpair;
  c->old_R = L.R;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->keep_state_ready = true;
  return NSN_OK;
}

// After the rebuild: lam_prev of the new build from the kept one -- contact
// rows by key (body pair and point on a; against the world also the normal,
// which is the plane's, so that a vertex touching two planes keeps one
// multiplier per plane), joint and tet rows by position when
// their counts did not change; rows without a match start from zero (a new
// contact has no previous-step multiplier).  The host computes the map from
// new to old internal rows; a kernel gathers.
template <typename T>
nsn_status restore_from_keep(nsn_ctx *c, const std::vector<nsn_contact> &old_contacts, int old_nj, int old_nt) {
  Dev<T> &D = dev<T>(c);
  const Layout &L = c->L;
  const HostScene &S = c->scene;
  if (L.R == 0 || !c->keep_lam) return NSN_OK;
  // map[ABI row] = old internal row (-1: none), built in ABI order (the
  // collider emits contacts by body, so the lookups walk the buckets in order)
  int *map = c->stage.take<int>(L.R);
  if (!map) return fail(c, NSN_ERR_OUT_OF_MEMORY, "pinned staging of the multiplier map");
  std::fill(map, map + L.R, -1);
  // the old contacts bucketed by body a + 1 (a = -1: the world), their keys
  // stored in bucket order so that each lookup scans a short contiguous run
  const int onc = int(old_contacts.size());
  const int nb = int(S.kind.size());
  // (a stable counting sort on host threads; end[s] = the old contacts with
  // key <= s: bucket s is list[end[s - 1] .. end[s]))
  std::vector<int> &end = c->key_end, &list = c->key_list, &bkey = c->key_k;
  order_by(onc, nb + 1, [&](int i) { return old_contacts[i].body_a + 1; }, list, bkey, c->key_cnt);
  end.assign(size_t(nb) + 2, 0);
  {
    const int nth = layout_threads(onc);
    parallel_for_threads(nth, [&](int h) {
      const int i0 = int((long long)onc * h / nth), i1 = int((long long)onc * (h + 1) / nth);
      for (int i = i0; i < i1; i++) {
        const int kk = bkey[list[i]];
        if (i == onc - 1 || bkey[list[i + 1]] != kk) end[kk] = i + 1;
      }
    });
  }
  for (int s = 1; s <= nb + 1; s++) end[s] = std::max(end[s], end[size_t(s) - 1]);
  std::vector<ContactKeyRec> &ok = c->okeys;
  ok.resize(onc);
  {
    const int nth = layout_threads(onc);
    const int ncinv = int(c->old_cinv.size());
    parallel_for_threads(nth, [&](int h) {
      const int j0 = int((long long)onc * h / nth), j1 = int((long long)onc * (h + 1) / nth);
      for (int jj = j0; jj < j1; jj++) {
        const nsn_contact &r = old_contacts[list[jj]];
        ContactKeyRec &k = ok[jj];
        k.a = r.body_a; k.b = r.body_b;
        std::memcpy(k.p, r.pa, sizeof k.p);
        std::memcpy(k.n, r.n, sizeof k.n);
        k.idx = list[jj] < ncinv ? c->old_cinv[list[jj]] : -1;
      }
    });
  }
  const int nthm = layout_threads(L.nc);
  parallel_for_threads(nthm, [&](int k0) {
    const int c0 = int((long long)L.nc * k0 / nthm), c1 = int((long long)L.nc * (k0 + 1) / nthm);
    for (int cc = c0; cc < c1; cc++) {
      const nsn_contact &r = S.contacts[cc];
      const int sl = r.body_a + 1;
      if (sl < 0 || sl > nb) continue;
      uint32_t p[3], n[3];
      std::memcpy(p, r.pa, sizeof p);
      std::memcpy(n, r.n, sizeof n);
      for (int jj = sl == 0 ? 0 : end[sl - 1]; jj < end[sl]; jj++) {
        const ContactKeyRec &k = ok[jj];
        if (k.b == r.body_b && k.p[0] == p[0] && k.p[1] == p[1] && k.p[2] == p[2] && k.a == r.body_a &&
            (k.b >= 0 || (k.n[0] == n[0] && k.n[1] == n[1] && k.n[2] == n[2]))) {
          if (k.idx >= 0)
            for (int q = 0; q < 3; q++) map[3 * cc + q] = 3 * k.idx + q;
          break;
        }
      }
    }
  });
  if (old_nj == L.nj && int(c->old_jinv.size()) == L.nj)
    for (int a = 0; a < L.nj; a++)
      for (int q = 0; q < 5; q++) map[3 * L.nc + 5 * a + q] = 3 * c->old_nc + 5 * c->old_jinv[a] + q;
  if (old_nt == L.nt && old_nj == L.nj && int(c->old_tinv.size()) == L.nt)
    for (int b = 0; b < L.nt; b++)
      for (int q = 0; q < 3; q++) map[L.tb_abi[b] + q] = c->old_Rpair + 3 * c->old_tinv[b] + q;
  // the map goes to the device through the entry scratch t2 (rewritten by
  // every evaluation before it is read)
  int *dmap = reinterpret_cast<int *>(D.t2);
  CUDA_TRY(c, cudaMemcpyAsync(dmap, map, sizeof(int) * L.R, cudaMemcpyHostToDevice, c->stream));
  k_gather_lam<T><<<clampb(cdiv(L.R, 256), D.max_blk), 256, 0, c->stream>>>(D.lam_prev, static_cast<const T *>(c->keep_lam),
                                                                         dmap, D.row_abi_dev, L.R);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaMemsetAsync(D.t2, 0, sizeof(T) * std::max(2 * L.Rpair + 12 * L.nt, 1), c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return NSN_OK;
}

nsn_status ensure_built(nsn_ctx *c) {
  if (!c->dirty) return NSN_OK;
  for (int k = NSN_PHASE_SAVE; k <= NSN_PHASE_RESTORE; k++) c->phase_ms[k] = 0.0;
  double t0 = now_ms();
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  const int nb = int(c->scene.kind.size());
  // the bodies did not change: state and multipliers stay on the device
  const bool keep = c->dmem && c->built_nb > 0 && c->built_nb == nb;
  c->keep_state_ready = false;
  if (keep) {
    nsn_status sk = c->cfg.precision == NSN_FP64 ? keep_for_rebuild<double>(c) : keep_for_rebuild<float>(c);
    if (sk != NSN_OK) return sk;
  } else if (c->dmem && c->built_nb > 0) {
    // bodies were added: the state of those already built comes back to the
    // host scene (multipliers start from zero)
    const int nb0 = c->built_nb;
    std::vector<float> pos(3 * nb0), quat(4 * nb0), vel(3 * nb0), om(3 * nb0);
    c->dirty = false;
    nsn_status s0 = state_io(c, false, false, nullptr, nullptr, nullptr, nullptr, pos.data(), quat.data(), vel.data(), om.data());
    c->dirty = true;
    if (s0 != NSN_OK) return s0;
    std::copy(pos.begin(), pos.end(), c->scene.pos.begin());
    std::copy(quat.begin(), quat.end(), c->scene.quat.begin());
    std::copy(vel.begin(), vel.end(), c->scene.vel.begin());
    std::copy(om.begin(), om.end(), c->scene.omega.begin());
  }
  phase_tick(c, NSN_PHASE_SAVE, t0);
  nsn_status s = build_layout(c);
  if (s != NSN_OK) return s;
  phase_tick(c, NSN_PHASE_LAYOUT, t0);
  s = c->cfg.precision == NSN_FP64 ? build_device<double>(c) : build_device<float>(c);
  if (s != NSN_OK) return s;
  phase_tick(c, NSN_PHASE_UPLOAD, t0);
  if (keep) {
    s = c->cfg.precision == NSN_FP64 ? restore_from_keep<double>(c, c->built_contacts, c->built_nj, c->built_nt)
                                     : restore_from_keep<float>(c, c->built_contacts, c->built_nj, c->built_nt);
    if (s != NSN_OK) return s;
  }
  phase_tick(c, NSN_PHASE_RESTORE, t0);
  c->dirty = false;
  c->built_nb = nb;
  {   // the contacts the device holds, for the next rebuild's key matching (copied on host threads)
    const std::vector<nsn_contact> &src = c->scene.contacts;
    std::vector<nsn_contact> &dst = c->built_contacts;
    const size_t n = src.size();
    dst.resize(n);
    const int nth = layout_threads((long long)n);
    parallel_for_threads(nth, [&](int h) {
      const size_t i0 = n * size_t(h) / size_t(nth), i1 = n * size_t(h + 1) / size_t(nth);
      if (i1 > i0) std::memcpy(dst.data() + i0, src.data() + i0, sizeof(nsn_contact) * (i1 - i0));
    });
  }
  c->built_nj = int(c->scene.joints.size());
  c->built_nt = c->L.nt;
  return NSN_OK;
}

nsn_status mlp_ensure(nsn_ctx *c, int rows_needed);

// The step as one CUDA graph: prefix, a conditional WHILE node for the Newton
// loop whose body holds a conditional WHILE node for the CR loop, suffix.
// The loop-control kernels set each node's condition on the device, so a step
// runs only the iterations it needs (islands that stop early, CR stopped by
// its tolerance); both loops stay bounded by their caps.
template <typename T>
nsn_status capture_step(nsn_ctx *c, Dev<T> &D) {
  cudaStream_t st = c->stream;
  const int N = c->cfg.newton_iters, M = c->cfg.cr_iters;
  Launcher<T> Lr{c, D, st};
  cudaGraph_t g = nullptr;
  CUDA_TRY(c, cudaGraphCreate(&g, 0));
  struct GraphGuard { cudaGraph_t g; ~GraphGuard() { if (g) cudaGraphDestroy(g); } } guard{g};
  auto capture = [&](cudaGraph_t graph, const std::vector<cudaGraphNode_t> &in, auto &&fn, int &kernels,
                     std::vector<cudaGraphNode_t> &out) -> cudaError_t {
    cudaError_t e = cudaStreamBeginCaptureToGraph(st, graph, in.empty() ? nullptr : in.data(), nullptr, in.size(),
                                                  cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const int before = Lr.count;
    fn();
    kernels = Lr.count - before;
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t *d = nullptr;
    size_t nd = 0;
    e = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &d, nullptr, &nd);
    if (e == cudaSuccess) out.assign(d, d + nd);
    cudaGraph_t gout = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(st, &gout);
    return e != cudaSuccess ? e : e2;
  };
  auto while_node = [&](cudaGraph_t graph, const std::vector<cudaGraphNode_t> &in, cudaGraphConditionalHandle h,
                        cudaGraphNode_t &node, cudaGraph_t &body) -> cudaError_t {
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    std::memset(raw, 0, sizeof raw);
    cudaGraphNodeParams &p = *reinterpret_cast<cudaGraphNodeParams *>(raw);
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaError_t e = cudaGraphAddNode(&node, graph, in.empty() ? nullptr : in.data(), nullptr, in.size(), &p);
    if (e == cudaSuccess) body = p.conditional.phGraph_out[0];
    return e;
  };
  c->seg = nsn_ctx::Segments();
  std::vector<cudaGraphNode_t> deps, tmp;
  CUDA_TRY(c, capture(g, deps, [&] { Lr.prefix(); }, c->seg.prefix, deps));
  if (N > 0) {
    cudaGraphConditionalHandle hN = 0, hC = 0;
    CUDA_TRY(c, cudaGraphConditionalHandleCreate(&hN, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNode_t nN;
    cudaGraph_t bN = nullptr;
    CUDA_TRY(c, while_node(g, deps, hN, nN, bN));
    const bool has_cr = D.R && M > 0 && D.streamed;
    if (has_cr) CUDA_TRY(c, cudaGraphConditionalHandleCreate(&hC, bN, 0, 0));
    D.hN = hN;
    D.hC = hC;
    std::vector<cudaGraphNode_t> body_deps;
    cudaError_t e = capture(bN, {}, [&] { Lr.newton_head(M); }, c->seg.head, body_deps);
    if (e == cudaSuccess && has_cr) {
      cudaGraphNode_t nC;
      cudaGraph_t bC = nullptr;
      e = while_node(bN, body_deps, hC, nC, bC);
      if (e == cudaSuccess) e = capture(bC, {}, [&] { Lr.cr_body(IT_DEV, M); }, c->seg.cr, tmp);
      body_deps.assign(1, nC);
    }
    if (e == cudaSuccess) e = capture(bN, body_deps, [&] { Lr.newton_tail(N); }, c->seg.tail, tmp);
    D.hN = 0;
    D.hC = 0;
    if (e != cudaSuccess) return fail(c, NSN_ERR_CUDA, "graph capture (Newton / CR loops): %s", cudaGetErrorString(e));
    deps.assign(1, nN);
  }
  CUDA_TRY(c, capture(g, deps, [&] { Lr.suffix(); }, c->seg.suffix, tmp));
  const cudaError_t e = cudaGraphInstantiate(&c->graph, g, 0);
  if (e != cudaSuccess) return fail(c, NSN_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return NSN_OK;
}

template <typename T>
nsn_status run_steps(nsn_ctx *c, int nsteps) {
  Dev<T> &D = dev<T>(c);
  cudaStream_t st = c->stream;
  D.warm = c->warm_mode;
  D.pscale_on = c->warm_mode == NSN_WARM_LEARNED && c->warm_precond ? 1 : 0;
  if (c->warm_mode == NSN_WARM_LEARNED) {
    if (!c->mlp.ready) return fail(c, NSN_ERR_BAD_STATE, "learned warm start without network parameters (nsn_mlp_set_params)");
    nsn_status s = mlp_ensure(c, D.nc);
    if (s != NSN_OK) return s;
  }
  // decision log: sized for the current layout, its pointers captured with the step
  const size_t dlog_need = size_t(c->dlog_iters) * (size_t(D.R) + 3 * size_t(D.ni));
  if (c->dlog_iters > 0 && (dlog_need > c->dlog_bytes || !c->dlog_buf)) {
    if (c->dlog_buf) cudaFree(c->dlog_buf);
    c->dlog_buf = nullptr;
    c->dlog_bytes = 0;
    if (cudaMalloc(&c->dlog_buf, std::max<size_t>(dlog_need, 1)) != cudaSuccess)
      return fail(c, NSN_ERR_OUT_OF_MEMORY, "decision log of %zu bytes", dlog_need);
    c->dlog_bytes = dlog_need;
  }
  unsigned char *want = c->dlog_iters > 0 ? c->dlog_buf : nullptr;
  if (D.dlog != want + (want ? 2 * size_t(c->dlog_iters) * D.ni : 0) || D.dlog_iters != c->dlog_iters) {
    // layout: CR counts (uint16, first for alignment), row codes, island codes
    D.dlog_cr = want ? reinterpret_cast<unsigned short *>(want) : nullptr;
    D.dlog = want ? want + 2 * size_t(c->dlog_iters) * D.ni : nullptr;
    D.dlog_ls = want ? D.dlog + size_t(c->dlog_iters) * D.R : nullptr;
    D.dlog_iters = want ? c->dlog_iters : 0;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  }
  c->phase_ms[NSN_PHASE_CAPTURE] = 0.0;
  if (!c->ev0) CUDA_TRY(c, cudaEventCreate(&c->ev0));
  if (!c->ev1) CUDA_TRY(c, cudaEventCreate(&c->ev1));
  CUDA_TRY(c, cudaEventRecord(c->ev0, st));
  if (c->cfg.use_graph) {
    if (!c->graph) {
      double t0 = now_ms();
      nsn_status s = capture_step<T>(c, D);
      if (s != NSN_OK) return s;
      phase_tick(c, NSN_PHASE_CAPTURE, t0);
    }
    for (int s = 0; s < nsteps; s++) {
      if (D.dlog) CUDA_TRY(c, cudaMemsetAsync(D.dlog_cr, 0xff, dlog_need, st));
      CUDA_TRY(c, cudaGraphLaunch(c->graph, st));
    }
  } else {
    for (int s = 0; s < nsteps; s++) {
      if (D.dlog) CUDA_TRY(c, cudaMemsetAsync(D.dlog_cr, 0xff, dlog_need, st));
      Launcher<T> Lr{c, D, st};
      Lr.step();
      c->launches_per_step = Lr.count;
    }
    CUDA_TRY(c, cudaGetLastError());
  }
  CUDA_TRY(c, cudaEventRecord(c->ev1, st));
  // stats of the last step
  Flags fl;
  Scalars sc;
  CUDA_TRY(c, cudaMemcpyAsync(&fl, D.fl, sizeof(Flags), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaMemcpyAsync(&sc, D.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->last.newton_done = fl.newton_count;
  c->last.cr_total = fl.cr_count;
  c->last.merit0 = sc.merit0;
  c->last.merit_final = sc.merit_final;
  c->last.ms = ms;
  c->last_newton_n = fl.newton_n;
  c->best_restored = D.best ? fl.best_restored : 0;
  c->kept_buf = fl.newton_n & 1;   // entries of the final evaluation
  D.pscale_on = 0;                 // the linearize / solve / apply paths use the Jacobi preconditioner
  if (c->cfg.use_graph)
    c->launches_per_step = c->seg.prefix + fl.newton_n * (c->seg.head + c->seg.tail) + fl.cr_exec * c->seg.cr +
                           c->seg.suffix;
  if (!std::isfinite(c->last.merit_final)) return fail(c, NSN_ERR_NONFINITE, "merit is not finite");
  if (c->warm_mode == NSN_WARM_LEARNED) return mlp_check(c, st);
  return NSN_OK;
}

bool valid_cfg(const nsn_config *cfg) {
  return cfg && cfg->h > 0 && cfg->newton_iters >= 0 && cfg->newton_iters < 1000 && cfg->cr_iters >= 0 &&
         cfg->damping > 0 && cfg->damping <= 1 && cfg->eps >= 0 && cfg->tol_rel >= 0 &&
         (cfg->precision == NSN_FP32 || cfg->precision == NSN_FP64) && (cfg->ncp == 0 || cfg->ncp == 1) &&
         cfg->rscale >= 0 && cfg->rscale <= 2 && (cfg->cone_project == 0 || cfg->cone_project == 1) &&
         (cfg->island_stop == 0 || cfg->island_stop == 1) && (cfg->cr_resident == 0 || cfg->cr_resident == 1) &&
         (cfg->line_search == 0 || cfg->line_search == 1) && (cfg->best_iterate == 0 || cfg->best_iterate == 1) &&
         (cfg->best_iterate == 0 || cfg->island_stop == 1);
}

template <typename T>
nsn_status do_linearize(nsn_ctx *c, int n_before) {
  Dev<T> &D = dev<T>(c);
  cudaStream_t st = c->stream;
  const int nbt = D.nr + D.np;
  T *bk = reinterpret_cast<T *>(c->d_backup);
  if (nbt) k_backup_state<T><<<cdiv(nbt, 128), 128, 0, st>>>(D, bk, 0);
  blocks_all_on(D, st);
  Launcher<T> Lr{c, D, st};
  Lr.begin();
  for (int n = 0; n < n_before; n++) {
    Lr.linearize_at(n);
    Lr.cr(c->cfg.cr_iters, n & 1);
    Lr.newton_update(n);
  }
  Lr.linearize_at(n_before);
  if (nbt) k_backup_state<T><<<cdiv(nbt, 128), 128, 0, st>>>(D, bk, 1);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaStreamSynchronize(st));
  c->linearized = true;
  return NSN_OK;
}

template <typename T>
__global__ void k_from_double(T *dst, const double *src, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = T(src[i]);
}
template <typename T>
__global__ void k_to_double(double *dst, const T *src, int n, int invert) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = invert ? 1.0 / double(src[i]) : double(src[i]);
}

template <typename T>
nsn_status copy_out(nsn_ctx *c, const T *src, int n, double *host, int invert = 0) {
  if (!host || n <= 0) return NSN_OK;
  double *tmp;
  CUDA_TRY(c, cudaMallocAsync(&tmp, sizeof(double) * n, c->stream));
  k_to_double<T><<<cdiv(n, 256), 256, 0, c->stream>>>(tmp, src, n, invert);
  CUDA_TRY(c, cudaMemcpyAsync(host, tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaFreeAsync(tmp, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return NSN_OK;
}

// a per-row vector in the caller's (ABI) row order
template <typename T>
nsn_status copy_out_rows(nsn_ctx *c, const T *src, double *host, int invert = 0) {
  const Layout &L = c->L;
  if (!host || L.R <= 0) return NSN_OK;
  std::vector<double> tmp(L.R);
  nsn_status s = copy_out<T>(c, src, L.R, tmp.data(), invert);
  if (s != NSN_OK) return s;
  for (int i = 0; i < L.R; i++) host[L.row_abi[i]] = tmp[i];
  return NSN_OK;
}

template <typename T>
nsn_status do_apply(nsn_ctx *c, const double *x, double *y) {
  Dev<T> &D = dev<T>(c);
  cudaStream_t st = c->stream;
  const int R = D.R;
  if (R == 0) return NSN_OK;
  double *tmp;
  std::vector<double> xi(R), yi(R);
  for (int i = 0; i < R; i++) xi[i] = x[c->L.row_abi[i]];
  CUDA_TRY(c, cudaMallocAsync(&tmp, sizeof(double) * R, st));
  CUDA_TRY(c, cudaMemcpyAsync(tmp, xi.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
  k_from_double<T><<<cdiv(R, 256), 256, 0, st>>>(D.z, tmp, R);
  CUDA_TRY(c, cudaMemsetAsync(D.fl, 0, sizeof(Flags), st));
  Launcher<T> Lr{c, D, st};
  Lr.body(BM_APPLY, D.z, c->lin_buf, 0, 1);
  Lr.rows(RM_APPLY, 1);
  k_to_double<T><<<cdiv(R, 256), 256, 0, st>>>(tmp, D.Az, R, 0);
  CUDA_TRY(c, cudaMemcpyAsync(yi.data(), tmp, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaFreeAsync(tmp, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  for (int i = 0; i < R; i++) y[c->L.row_abi[i]] = yi[i];
  return NSN_OK;
}

// du in body order from the BM_UPDATE formula without committing: computed on
// the host from g, H~^-1 blocks and J^T dl gathered through the apply path.
template <typename T>
nsn_status do_solve(nsn_ctx *c, int iters, double *dl, double *du) {
  Dev<T> &D = dev<T>(c);
  cudaStream_t st = c->stream;
  CUDA_TRY(c, cudaMemsetAsync(D.fl, 0, sizeof(Flags), st));
  blocks_all_on(D, st);
  if (D.R) {
    k_cr_init<T><<<D.nblk_upd, BLOCK, 0, st>>>(D);
    // res0 for the scalar kernel
    Launcher<T> Lr{c, D, st};
    Lr.cr(iters, c->lin_buf);
  }
  CUDA_TRY(c, cudaGetLastError());
  if (dl) { nsn_status s = copy_out_rows<T>(c, D.x, dl); if (s) return s; }
  if (du) {
    // du = H~^-1 (h J^T dl - g): reuse the apply body pass on x to get y = H~^-1 J^T x
    // per body into the per-entry scratch is not body-ordered, so do it on the host.
    const Layout &L = c->L;
    const int nb = int(c->scene.kind.size());
    std::vector<double> x(D.R);
    auto row_of = [&](int slot) { return slot < 2 * L.Rpair ? slot / 2 : L.Rpair + (slot - 2 * L.Rpair) / 4; };
    if (D.R) { nsn_status s = copy_out<T>(c, D.x, D.R, x.data()); if (s) return s; }
    std::vector<T> J6(size_t(6) * L.ER), J3(size_t(3) * L.EV);
    std::vector<T> g6(size_t(6) * L.nr), g3(size_t(3) * L.np), Iwi(size_t(6) * L.nr), hinv(size_t(3) * L.np), im(L.nr);
    int bufJ = -1;
    (void)bufJ;
    std::vector<RV4<T>> jA(L.ER);
    std::vector<RV2<T>> jB(L.ER);
    if (L.ER) {
      CUDA_TRY(c, cudaMemcpyAsync(jA.data(), D.ejA, sizeof(RV4<T>) * L.ER, cudaMemcpyDeviceToHost, st));
      CUDA_TRY(c, cudaMemcpyAsync(jB.data(), D.ejB, sizeof(RV2<T>) * L.ER, cudaMemcpyDeviceToHost, st));
    }
    for (int k = 0; k < 6; k++) {
      if (L.nr) {
        CUDA_TRY(c, cudaMemcpyAsync(g6.data() + size_t(k) * L.nr, D.rg[k], sizeof(T) * L.nr, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(c, cudaMemcpyAsync(Iwi.data() + size_t(k) * L.nr, D.rIwi[k], sizeof(T) * L.nr, cudaMemcpyDeviceToHost, st));
      }
    }
    if (L.nr) CUDA_TRY(c, cudaMemcpyAsync(im.data(), D.rinvm, sizeof(T) * L.nr, cudaMemcpyDeviceToHost, st));
    int lbuf = c->lin_buf;
    for (int k = 0; k < 3; k++) {
      if (L.EV) CUDA_TRY(c, cudaMemcpyAsync(J3.data() + size_t(k) * L.EV, D.ej3[lbuf][k], sizeof(T) * L.EV, cudaMemcpyDeviceToHost, st));
      if (L.np) {
        CUDA_TRY(c, cudaMemcpyAsync(g3.data() + size_t(k) * L.np, D.pg[k], sizeof(T) * L.np, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(c, cudaMemcpyAsync(hinv.data() + size_t(k) * L.np, D.phinv[k], sizeof(T) * L.np, cudaMemcpyDeviceToHost, st));
      }
    }
    CUDA_TRY(c, cudaStreamSynchronize(st));
    for (int q = 0; q < L.ER; q++) {
      const T v[6] = {jA[q].a, jA[q].b, jA[q].c, jA[q].d, jB[q].a, jB[q].b};
      for (int k = 0; k < 6; k++) J6[size_t(k) * L.ER + q] = v[k];
    }
    const double h = c->cfg.h;
    int off = 0;
    for (int i = 0; i < nb; i++) {
      int e = L.bmap[i];
      if (e >= 0) {
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int q = L.rseg[e]; q < L.rseg[e + 1]; q++)
          for (int k = 0; k < 6; k++) s[k] += double(J6[size_t(k) * L.ER + q]) * x[row_of(L.eslot[q])];
        double r[6];
        for (int k = 0; k < 6; k++) r[k] = h * s[k] - double(g6[size_t(k) * L.nr + e]);
        const T *S6 = nullptr;
        (void)S6;
        double Si[6];
        for (int k = 0; k < 6; k++) Si[k] = double(Iwi[size_t(k) * L.nr + e]);
        du[off + 0] = r[0] * double(im[e]); du[off + 1] = r[1] * double(im[e]); du[off + 2] = r[2] * double(im[e]);
        du[off + 3] = Si[0] * r[3] + Si[3] * r[4] + Si[4] * r[5];
        du[off + 4] = Si[3] * r[3] + Si[1] * r[4] + Si[5] * r[5];
        du[off + 5] = Si[4] * r[3] + Si[5] * r[4] + Si[2] * r[5];
        off += 6;
      } else {
        int p = -e - 2;
        double s[3] = {0, 0, 0};
        for (int q = L.vseg[p]; q < L.vseg[p + 1]; q++)
          for (int k = 0; k < 3; k++) s[k] += double(J3[size_t(k) * L.EV + q]) * x[row_of(L.eslot[L.ER + q])];
        for (int k = 0; k < 3; k++)
          du[off + k] = (h * s[k] - double(g3[size_t(k) * L.np + p])) * double(hinv[size_t(k) * L.np + p]);
        off += 3;
      }
    }
  }
  return NSN_OK;
}

template <typename T>
nsn_status do_system(nsn_ctx *c, double *b, double *diag, double *hvec, double *g) {
  Dev<T> &D = dev<T>(c);
  nsn_status s;
  if ((s = copy_out_rows<T>(c, D.b, b))) return s;
  if ((s = copy_out_rows<T>(c, D.P, diag, 1))) return s;
  if ((s = copy_out_rows<T>(c, D.hv, hvec))) return s;
  if (g) {
    const Layout &L = c->L;
    std::vector<double> g6(size_t(6) * L.nr), g3(size_t(3) * L.np);
    for (int k = 0; k < 6; k++)
      if ((s = copy_out<T>(c, D.rg[k], L.nr, g6.data() + size_t(k) * L.nr))) return s;
    for (int k = 0; k < 3; k++)
      if ((s = copy_out<T>(c, D.pg[k], L.np, g3.data() + size_t(k) * L.np))) return s;
    int off = 0;
    for (size_t i = 0; i < c->scene.kind.size(); i++) {
      int e = L.bmap[i];
      if (e >= 0) { for (int k = 0; k < 6; k++) g[off + k] = g6[size_t(k) * L.nr + e]; off += 6; }
      else { int p = -e - 2; for (int k = 0; k < 3; k++) g[off + k] = g3[size_t(k) * L.np + p]; off += 3; }
    }
  }
  return NSN_OK;
}

}  // namespace

namespace {
// k_cr_resident timed alone at the first Newton iteration of a zero start
// (every resident island continues), the committed state kept
template <typename T>
nsn_status do_time_resident(nsn_ctx *c, int iters, float *ms, double *work4) {
  Dev<T> &D = dev<T>(c);
  cudaStream_t st = c->stream;
  if (!D.res_on) return NSN_ERR_INVALID_ARG;
  nsn_status s = do_linearize<T>(c, 0);
  if (s != NSN_OK) return s;
  cudaEvent_t e[2];
  for (auto &x : e) CUDA_TRY(c, cudaEventCreate(&x));
  const int M = c->cfg.cr_iters;
  Flags *f = D.fl;
  const size_t wofs = offsetof(Flags, res_rowit);
  Dev<T> Dw = D;
  Dw.res_work = 1;   // these launches count their work; the step's do not
  float tot = 0.f;
  Flags fl{};
  for (int i = 0; i <= iters; i++) {   // launch 0 is a warm-up
    CUDA_TRY(c, cudaMemsetAsync(&f->res_next, 0, sizeof(int), st));
    CUDA_TRY(c, cudaMemsetAsync(&f->cr_res_max, 0, sizeof(int), st));
    CUDA_TRY(c, cudaMemsetAsync(reinterpret_cast<char *>(f) + wofs, 0, 3 * sizeof(unsigned long long), st));
    CUDA_TRY(c, cudaEventRecord(e[0], st));
    k_cr_resident<T><<<D.nblk_res, RES_THREADS, D.res_smem, st>>>(Dw, M);
    CUDA_TRY(c, cudaEventRecord(e[1], st));
    CUDA_TRY(c, cudaMemcpyAsync(&fl, f, sizeof(Flags), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    float t = 0.f;
    CUDA_TRY(c, cudaEventElapsedTime(&t, e[0], e[1]));
    if (i > 0) tot += t;
  }
  for (auto &x : e) cudaEventDestroy(x);
  if (ms) *ms = iters > 0 ? tot / iters : 0.f;
  if (work4) {
    work4[0] = double(fl.n_list_res);
    work4[1] = double(fl.res_rowit);
    work4[2] = double(fl.res_entit);
    work4[3] = double(fl.res_bodit);
  }
  c->linearized = false;
  return NSN_OK;
}

template <typename T>
nsn_status do_time_operator(nsn_ctx *c, int iters, float *ms_body, float *ms_row) {
  Dev<T> &D = dev<T>(c);
  cudaStream_t st = c->stream;
  cudaEvent_t e[3];
  for (auto &x : e) CUDA_TRY(c, cudaEventCreate(&x));
  CUDA_TRY(c, cudaMemsetAsync(D.fl, 0, sizeof(Flags), st));
  // island mode: time the apply with every island taking part
  if (D.isl_on && D.ni) {
    CUDA_TRY(c, cudaMemsetAsync(D.isl.crdone, 0, sizeof(int) * D.ni, st));
    CUDA_TRY(c, cudaMemsetAsync(D.fl_row, 1, size_t(D.R) / BLOCK + 1, st));
    CUDA_TRY(c, cudaMemsetAsync(D.fl_br, 1, size_t(D.nr) / (BLOCK / 16) + 1, st));
    CUDA_TRY(c, cudaMemsetAsync(D.fl_bp, 1, size_t(D.np) / (BLOCK / 16) + 1, st));
  }
  Launcher<T> Lr{c, D, st};
  double tb = 0.0, tr = 0.0;
  const int buf = c->kept_buf < 0 ? 0 : c->kept_buf;  // entries written by the final evaluation of the last step
  for (int i = 0; i < iters; i++) {
    CUDA_TRY(c, cudaEventRecord(e[0], st));
    Lr.body(BM_APPLY, D.z, buf, 0, 1);
    CUDA_TRY(c, cudaEventRecord(e[1], st));
    Lr.rows(RM_APPLY, 1);
    CUDA_TRY(c, cudaEventRecord(e[2], st));
    CUDA_TRY(c, cudaEventSynchronize(e[2]));
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, e[0], e[1]);
    cudaEventElapsedTime(&b, e[1], e[2]);
    tb += a; tr += b;
  }
  for (auto &x : e) cudaEventDestroy(x);
  if (D.isl_on && D.ni) CUDA_TRY(c, cudaMemsetAsync(D.isl.acc, 0, sizeof(double) * ISL_ACC * D.ni, st));
  CUDA_TRY(c, cudaGetLastError());
  if (ms_body) *ms_body = float(tb / std::max(iters, 1));
  if (ms_row) *ms_row = float(tr / std::max(iters, 1));
  return NSN_OK;
}

}  // namespace


// ------------------------------------------------------------------------------------
// learned warm start: network workspace, inference and training

namespace {

template <typename X>
nsn_status dalloc(nsn_ctx *c, X **p, size_t n) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), sizeof(X) * (n ? n : 1));
  if (e != cudaSuccess) return fail(c, NSN_ERR_OUT_OF_MEMORY, "cudaMalloc: %s", cudaGetErrorString(e));
  return NSN_OK;
}

void mlp_free(MlpState &m) {
  void *ptrs[] = {m.pf, m.gr, m.m, m.v, m.pb, m.xb, m.a1b, m.a2b, m.a3b, m.dyb, m.dzb, m.a1f, m.a2f, m.a3f,
                  m.y, m.dyf, m.da, m.dzf, m.lpart, m.X, m.Y, m.err};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  m = MlpState();
}

constexpr int kMlpChunk = 65536;

nsn_status mlp_workspace(nsn_ctx *c, int cap) {
  MlpState &m = c->mlp;
  if (cap <= m.cap) return NSN_OK;
  nsn_status s;
  const size_t H = size_t(cap) * mlp::NH;
  if ((s = dalloc(c, &m.xb, size_t(cap) * mlp::NIN)) || (s = dalloc(c, &m.a1b, H)) || (s = dalloc(c, &m.a2b, H)) ||
      (s = dalloc(c, &m.a3b, H)) || (s = dalloc(c, &m.dzb, H)) || (s = dalloc(c, &m.a1f, H)) ||
      (s = dalloc(c, &m.a2f, H)) || (s = dalloc(c, &m.a3f, H)) || (s = dalloc(c, &m.da, H)) ||
      (s = dalloc(c, &m.dzf, H)) || (s = dalloc(c, &m.y, size_t(cap) * mlp::NOUT)) ||
      (s = dalloc(c, &m.dyf, size_t(cap) * mlp::NOUT)) || (s = dalloc(c, &m.dyb, size_t(cap) * mlp::NOUT)) ||
      (s = dalloc(c, &m.lpart, 1024)))
    return s;
  m.cap = cap;
  return NSN_OK;
}

template <bool TA, bool TB>
void gemm(const __nv_bfloat16 *A, const __nv_bfloat16 *B, const float *bias, float *Cf, __nv_bfloat16 *Cb, int M, int N,
          int K, int lda, int ldb, int ldc, int relu, cudaStream_t st) {
  dim3 grid(cdiv(N, mlp::TN), cdiv(M, mlp::TM));
  mlp::k_gemm<TA, TB><<<grid, 128, 0, st>>>(A, B, bias, Cf, Cb, M, N, K, lda, ldb, ldc, relu);
}

// forward pass of n rows (n <= cap); keeps FP32 post-activations when train
void mlp_forward_rows(MlpState &m, const float *X, int n, float *Y, bool train, cudaStream_t st) {
  using namespace mlp;
  k_to_bf16<<<cdiv(size_t(n) * NIN, 256), 256, 0, st>>>(X, m.xb, n * NIN);
  gemm<false, true>(m.xb, m.pb + OFF_W1, m.pf + OFF_B1, train ? m.a1f : nullptr, m.a1b, n, NH, NIN, NIN, NIN, NH, 1, st);
  gemm<false, true>(m.a1b, m.pb + OFF_W2, m.pf + OFF_B2, train ? m.a2f : nullptr, m.a2b, n, NH, NH, NH, NH, NH, 1, st);
  gemm<false, true>(m.a2b, m.pb + OFF_W3, m.pf + OFF_B3, train ? m.a3f : nullptr, m.a3b, n, NH, NH, NH, NH, NH, 1, st);
  gemm<false, true>(m.a3b, m.pb + OFF_W4, m.pf + OFF_B4, Y, nullptr, n, NOUT, NH, NH, NH, NOUT, 0, st);
}

nsn_status mlp_ensure(nsn_ctx *c, int rows_needed) {
  MlpState &m = c->mlp;
  nsn_status s = mlp_workspace(c, kMlpChunk);
  if (s != NSN_OK) return s;
  if (rows_needed > m.ncap) {
    if ((s = dalloc(c, &m.X, size_t(rows_needed) * mlp::NIN)) || (s = dalloc(c, &m.Y, size_t(rows_needed) * mlp::NOUT)))
      return s;
    m.ncap = rows_needed;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  }
  return NSN_OK;
}

// inference: one tcgen05 kernel (weights resident in shared memory, the
// accumulator in TMEM), persistent over tiles of 128 rows, two CTAs per SM
nsn_status mlp_infer(nsn_ctx *c, const float *X, int n, float *Y, cudaStream_t st) {
  MlpState &m = c->mlp;
  if (n <= 0) return NSN_OK;
  const size_t smem = sizeof(mlp::TcSmem);
  static bool attr_set = false;
  if (!attr_set) {
    CUDA_TRY(c, cudaFuncSetAttribute(mlp::k_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    attr_set = true;
  }
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = cdiv(n, mlp::TC_M);
  const int xvec = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  mlp::k_forward_tc<<<std::min(tiles, 2 * nsm), mlp::TC_THREADS, smem, st>>>(X, n, xvec, m.pb, m.pf, Y, m.err);
  return NSN_OK;
}

// the inference kernel's time-out flag (read and cleared; synchronises st)
nsn_status mlp_check(nsn_ctx *c, cudaStream_t st) {
  MlpState &m = c->mlp;
  if (!m.err) return NSN_OK;
  int e = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&e, m.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  if (!e) return NSN_OK;
  CUDA_TRY(c, cudaMemsetAsync(m.err, 0, sizeof(int), st));
  return fail(c, NSN_ERR_TIMEOUT, "network inference: a tensor-core completion wait timed out");
}

nsn_status mlp_train(nsn_ctx *c, const float *X, const float *Tg, const float *w, int n, float lr, float *loss) {
  using namespace mlp;
  MlpState &m = c->mlp;
  cudaStream_t st = c->stream;
  nsn_status s = mlp_workspace(c, std::max(n, 64));
  if (s != NSN_OK) return s;
  mlp_forward_rows(m, X, n, m.y, true, st);
  const int nb = std::min(cdiv(size_t(n) * NOUT, 256), 1024);
  k_loss_grad<<<nb, 256, 0, st>>>(m.y, Tg, w, m.dyb, m.dyf, n, m.lpart);
  float *g = m.gr;
  const int cs = 128;
  // layer 4
  gemm<true, false>(m.dyb, m.a3b, nullptr, g + OFF_W4, nullptr, NOUT, NH, n, NOUT, NH, NH, 0, st);
  k_colsum<<<1, cs, 0, st>>>(m.dyf, g + OFF_B4, n, NOUT);
  gemm<false, false>(m.dyb, m.pb + OFF_W4, nullptr, m.da, nullptr, n, NH, NOUT, NOUT, NH, NH, 0, st);
  // layer 3
  k_relu_back<<<cdiv(size_t(n) * NH, 256), 256, 0, st>>>(m.da, m.a3f, m.dzb, m.dzf, n * NH);
  gemm<true, false>(m.dzb, m.a2b, nullptr, g + OFF_W3, nullptr, NH, NH, n, NH, NH, NH, 0, st);
  k_colsum<<<1, cs, 0, st>>>(m.dzf, g + OFF_B3, n, NH);
  gemm<false, false>(m.dzb, m.pb + OFF_W3, nullptr, m.da, nullptr, n, NH, NH, NH, NH, NH, 0, st);
  // layer 2
  k_relu_back<<<cdiv(size_t(n) * NH, 256), 256, 0, st>>>(m.da, m.a2f, m.dzb, m.dzf, n * NH);
  gemm<true, false>(m.dzb, m.a1b, nullptr, g + OFF_W2, nullptr, NH, NH, n, NH, NH, NH, 0, st);
  k_colsum<<<1, cs, 0, st>>>(m.dzf, g + OFF_B2, n, NH);
  gemm<false, false>(m.dzb, m.pb + OFF_W2, nullptr, m.da, nullptr, n, NH, NH, NH, NH, NH, 0, st);
  // layer 1
  k_relu_back<<<cdiv(size_t(n) * NH, 256), 256, 0, st>>>(m.da, m.a1f, m.dzb, m.dzf, n * NH);
  gemm<true, false>(m.dzb, m.xb, nullptr, g + OFF_W1, nullptr, NH, NIN, n, NH, NIN, NIN, 0, st);
  k_colsum<<<1, cs, 0, st>>>(m.dzf, g + OFF_B1, n, NH);
  if (lr > 0.f) {
    m.adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - std::pow(b1, float(m.adam_t)), bc2 = 1.f - std::pow(b2, float(m.adam_t));
    k_adam<<<cdiv(NPARAM, 256), 256, 0, st>>>(m.pf, g, m.m, m.v, m.pb, NPARAM, lr, b1, b2, 1e-8f, bc1, bc2);
  }
  CUDA_TRY(c, cudaGetLastError());
  if (loss) {
    float part[1024];
    CUDA_TRY(c, cudaMemcpyAsync(part, m.lpart, sizeof(float) * nb, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    double l = 0.0;
    for (int i = 0; i < nb; i++) l += part[i];
    *loss = float(l / n);
  }
  return NSN_OK;
}

template <typename T>
nsn_status do_features(nsn_ctx *c, float *X, float *Ytarget) {
  Dev<T> &D = dev<T>(c);
  if (!D.nc) return NSN_OK;
  if (X) k_contact_features<T><<<cdiv(D.nc, 128), 128, 0, c->stream>>>(D, X);
  if (Ytarget) k_contact_targets<T><<<cdiv(D.nc, 128), 128, 0, c->stream>>>(D, Ytarget);
  CUDA_TRY(c, cudaGetLastError());
  return NSN_OK;
}

}  // namespace

// =====================================================================================
// C ABI

extern "C" {

void nsn_default_config(nsn_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof *cfg);
  cfg->h = 1.0 / 60.0;
  cfg->gravity[2] = -9.81;
  cfg->newton_iters = 4;
  cfg->cr_iters = 20;
  cfg->damping = 0.75;
  cfg->eps = 1e-6;
  cfg->tol_rel = 0.0;
  cfg->cr_tol_mode = 0;
  cfg->ncp = NSN_NCP_FB;
  cfg->rscale = NSN_R_EFFMASS;
  cfg->geom_stiffness = NSN_GS_PARTICLES;
  cfg->precision = NSN_FP32;
  cfg->use_graph = 1;
  cfg->cone_project = 0;
  cfg->island_stop = 0;
  cfg->cr_resident = 1;
  cfg->res_max_rows = 384;
  cfg->line_search = 0;
}

nsn_status nsn_create(const nsn_config *cfg, void *stream, nsn_ctx **out) {
  if (!out) return NSN_ERR_INVALID_ARG;
  *out = nullptr;
  if (!valid_cfg(cfg)) return NSN_ERR_INVALID_ARG;
  nsn_ctx *c = new (std::nothrow) nsn_ctx();
  if (!c) return NSN_ERR_OUT_OF_MEMORY;
  c->cfg = *cfg;
  if (stream) c->stream = static_cast<cudaStream_t>(stream);
  else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return NSN_ERR_CUDA; }
    c->own_stream = true;
  }
  *out = c;   // the timing events are created by the first step
  return NSN_OK;
}

nsn_status nsn_destroy(nsn_ctx *c) {
  if (!c) return NSN_ERR_INVALID_ARG;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->dmem) cudaFree(c->dmem);
  mlp_free(c->mlp);
  if (c->dlog_buf) cudaFree(c->dlog_buf);
  if (c->col_state) cudaFree(c->col_state);
  if (c->col_body) cudaFree(c->col_body);
  if (c->col_f) cudaFree(c->col_f);
  if (c->col_found) cudaFree(c->col_found);
  c->stage.release();
  if (c->keep_state) cudaFree(c->keep_state);
  if (c->keep_lam) cudaFree(c->keep_lam);
  if (c->col_found_h) cudaFreeHost(c->col_found_h);
  if (c->col_f_h) cudaFreeHost(c->col_f_h);
  if (c->col_body_h) cudaFreeHost(c->col_body_h);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return NSN_OK;
}

const char *nsn_last_error(const nsn_ctx *c) { return c ? c->err.c_str() : "null context"; }

nsn_status nsn_add_bodies(nsn_ctx *c, int32_t n, const int32_t *kind, const float *pos, const float *quat,
                          const float *vel, const float *omega, const float *mass, const float *inertia,
                          int32_t *first_id) {
  if (!c) return NSN_ERR_INVALID_ARG;
  if (n < 0 || (n > 0 && (!kind || !pos || !vel || !mass))) return fail(c, NSN_ERR_INVALID_ARG, "add_bodies: null array");
  for (int i = 0; i < n; i++) {
    if (kind[i] != NSN_RIGID && kind[i] != NSN_PARTICLE) return fail(c, NSN_ERR_INVALID_ARG, "body %d: bad kind", i);
    if (!(mass[i] > 0.f) || !std::isfinite(mass[i])) return fail(c, NSN_ERR_INVALID_ARG, "body %d: mass must be > 0", i);
    if (kind[i] == NSN_RIGID) {
      if (!inertia) return fail(c, NSN_ERR_INVALID_ARG, "rigid bodies need inertia");
      for (int k = 0; k < 3; k++)
        if (!(inertia[3 * i + k] > 0.f)) return fail(c, NSN_ERR_INVALID_ARG, "body %d: inertia must be > 0", i);
    }
  }
  if (!finite_all(pos, size_t(3) * n) || !finite_all(vel, size_t(3) * n) ||
      (quat && !finite_all(quat, size_t(4) * n)) || (omega && !finite_all(omega, size_t(3) * n)))
    return fail(c, NSN_ERR_INVALID_ARG, "add_bodies: non-finite state");
  HostScene &S = c->scene;
  if (first_id) *first_id = int32_t(S.kind.size());
  for (int i = 0; i < n; i++) {
    S.kind.push_back(kind[i]);
    for (int k = 0; k < 3; k++) {
      S.pos.push_back(pos[3 * i + k]);
      S.vel.push_back(vel[3 * i + k]);
      S.omega.push_back(omega ? omega[3 * i + k] : 0.f);
      S.inertia.push_back(inertia && kind[i] == NSN_RIGID ? inertia[3 * i + k] : 1.f);
    }
    float q[4] = {1, 0, 0, 0};
    if (quat && kind[i] == NSN_RIGID) {
      double nn = 0;
      for (int k = 0; k < 4; k++) nn += double(quat[4 * i + k]) * quat[4 * i + k];
      if (!(std::fabs(nn - 1.0) < 1e-4)) return fail(c, NSN_ERR_INVALID_ARG, "body %d: quaternion is not unit", i);
      for (int k = 0; k < 4; k++) q[k] = quat[4 * i + k];
    }
    for (int k = 0; k < 4; k++) S.quat.push_back(q[k]);
    S.mass.push_back(mass[i]);
  }
  c->dirty = true;
  return NSN_OK;
}

nsn_status nsn_add_constraints(nsn_ctx *c, int32_t type, int32_t n, const void *records, int32_t *first_row) {
  if (!c) return NSN_ERR_INVALID_ARG;
  if (n < 0 || (n > 0 && !records)) return fail(c, NSN_ERR_INVALID_ARG, "add_constraints: null records");
  HostScene &S = c->scene;
  const int nb = int(S.kind.size());
  auto body_ok = [&](int id) { return id >= -1 && id < nb; };
  {
    // the device layout indexes rows and Jacobian entries with int32: the scene
    // after this call must keep 3 nc + 5 nj + 3 nt rows and 2 (3 nc + 5 nj) +
    // 12 nt entries below 2^31 (checked in int64 before anything is stored)
    const int64_t nc = int64_t(S.contacts.size()) + (type == NSN_CONTACT ? n : 0);
    const int64_t nj = int64_t(S.joints.size()) + (type == NSN_REVOLUTE || type == NSN_PRISMATIC ? n : 0);
    const int64_t nt = int64_t(S.tets.size()) + (type == NSN_TET_NH ? n : 0);
    const int64_t nl = int64_t(S.ltets.size()) + (type == NSN_TET_LINEAR ? n : 0);
    const int64_t rows = 3 * nc + 5 * nj + 3 * nt + 6 * nl, entries = 2 * (3 * nc + 5 * nj) + 12 * nt + 24 * nl;
    if (rows > INT32_MAX || entries > INT32_MAX)
      return fail(c, NSN_ERR_INVALID_ARG,
                  "add_constraints: the scene would hold %lld rows and %lld Jacobian entries (limit 2^31 - 1)",
                  (long long)rows, (long long)entries);
  }
  if (type == NSN_CONTACT) {
    const nsn_contact *r = static_cast<const nsn_contact *>(records);
    for (int i = 0; i < n; i++) {
      if (!body_ok(r[i].body_a) || !body_ok(r[i].body_b) || (r[i].body_a < 0 && r[i].body_b < 0) ||
          r[i].body_a == r[i].body_b)
        return fail(c, NSN_ERR_INVALID_ARG, "contact %d: bad body ids", i);
      double nn = double(r[i].n[0]) * r[i].n[0] + double(r[i].n[1]) * r[i].n[1] + double(r[i].n[2]) * r[i].n[2];
      if (!(std::fabs(nn - 1.0) < 1e-4) || !finite_all(r[i].pa, 3) || !finite_all(r[i].pb, 3) || !std::isfinite(r[i].d) ||
          !(r[i].mu >= 0.f))
        return fail(c, NSN_ERR_INVALID_ARG, "contact %d: bad geometry", i);
    }
    if (first_row) *first_row = 3 * int32_t(S.contacts.size());
    S.contacts.insert(S.contacts.end(), r, r + n);
  } else if (type == NSN_REVOLUTE || type == NSN_PRISMATIC) {
    const nsn_revolute *r = static_cast<const nsn_revolute *>(records);
    for (int i = 0; i < n; i++) {
      int a = r[i].body_a, b = r[i].body_b;
      if (!body_ok(a) || !body_ok(b) || (a < 0 && b < 0) || a == b) return fail(c, NSN_ERR_INVALID_ARG, "joint %d: bad body ids", i);
      if ((a >= 0 && S.kind[a] != NSN_RIGID) || (b >= 0 && S.kind[b] != NSN_RIGID))
        return fail(c, NSN_ERR_INVALID_ARG, "joint %d: joints connect rigid bodies", i);
      if (!(r[i].compliance >= 0.f)) return fail(c, NSN_ERR_INVALID_ARG, "joint %d: compliance < 0", i);
      if (type == NSN_PRISMATIC) {
        const double la = double(r[i].axis_a[0]) * r[i].axis_a[0] + double(r[i].axis_a[1]) * r[i].axis_a[1] +
                          double(r[i].axis_a[2]) * r[i].axis_a[2];
        const double lb = double(r[i].axis_b[0]) * r[i].axis_b[0] + double(r[i].axis_b[1]) * r[i].axis_b[1] +
                          double(r[i].axis_b[2]) * r[i].axis_b[2];
        if (!(la > 1e-12) || !(lb > 1e-12) || !finite_all(r[i].axis_a, 3) || !finite_all(r[i].axis_b, 3))
          return fail(c, NSN_ERR_INVALID_ARG, "joint %d: prismatic axes must be nonzero", i);
      }
    }
    if (first_row) *first_row = 5 * int32_t(S.joints.size());
    S.joints.insert(S.joints.end(), r, r + n);
    S.jkind.insert(S.jkind.end(), size_t(n), type == NSN_PRISMATIC ? 1 : 0);
  } else if (type == NSN_TET_NH || type == NSN_TET_LINEAR) {
    const nsn_tet *r = static_cast<const nsn_tet *>(records);
    for (int i = 0; i < n; i++) {
      for (int q = 0; q < 4; q++) {
        int v = r[i].v[q];
        if (v < 0 || v >= nb || S.kind[v] != NSN_PARTICLE) return fail(c, NSN_ERR_INVALID_ARG, "tet %d: vertex %d is not a particle", i, q);
        for (int p = 0; p < q; p++)
          if (r[i].v[p] == v) return fail(c, NSN_ERR_INVALID_ARG, "tet %d: repeated vertex", i);
      }
      double Dm[9];
      for (int row = 0; row < 3; row++)
        for (int k = 0; k < 3; k++) Dm[3 * row + k] = double(r[i].rest[k + 1][row]) - double(r[i].rest[0][row]);
      double det = Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
                   Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
      if (!(std::fabs(det) > 1e-18)) return fail(c, NSN_ERR_INVALID_ARG, "tet %d: degenerate rest shape", i);
      if (!(r[i].E > 0.f) || !(r[i].nu > 0.f && r[i].nu < 0.5f)) return fail(c, NSN_ERR_INVALID_ARG, "tet %d: bad material", i);
    }
    if (type == NSN_TET_NH) {
      if (first_row) *first_row = 3 * int32_t(S.tets.size());
      S.tets.insert(S.tets.end(), r, r + n);
    } else {
      if (first_row) *first_row = 6 * int32_t(S.ltets.size());
      S.ltets.insert(S.ltets.end(), r, r + n);
    }
  } else {
    return fail(c, NSN_ERR_INVALID_ARG, "unknown constraint type %d", type);
  }
  c->dirty = true;
  return NSN_OK;
}

nsn_status nsn_clear_contacts(nsn_ctx *c) {
  if (!c) return NSN_ERR_INVALID_ARG;
  c->scene.contacts.clear();
  c->dirty = true;
  return NSN_OK;
}

nsn_status nsn_counts(nsn_ctx *c, int32_t *n_bodies, int32_t *n_rows) {
  if (!c) return NSN_ERR_INVALID_ARG;
  if (n_bodies) *n_bodies = int32_t(c->scene.kind.size());
  if (n_rows)
    *n_rows = int32_t(3 * c->scene.contacts.size() + 5 * c->scene.joints.size() + 3 * c->scene.tets.size() +
                      6 * c->scene.ltets.size());
  return NSN_OK;
}

nsn_status nsn_step(nsn_ctx *c, int32_t nsteps, nsn_stats *stats) {
  if (!c || nsteps < 0) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  c->linearized = false;
  const double t0 = now_ms();
  s = c->cfg.precision == NSN_FP64 ? run_steps<double>(c, nsteps) : run_steps<float>(c, nsteps);
  c->phase_ms[NSN_PHASE_STEP] = now_ms() - t0 - c->phase_ms[NSN_PHASE_CAPTURE];

  if (stats) *stats = c->last;
  return s;
}

}  // extern "C"

nsn_status state_io(nsn_ctx *c, bool set, bool device, const float *ipos, const float *iquat,
                    const float *ivel, const float *iom, float *opos, float *oquat, float *ovel, float *oom) {
  if (!c) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  const int nb = int(c->scene.kind.size());
  if (!nb) return NSN_OK;
  cudaStream_t st = c->stream;
  float *stg = c->d_stage;
  float *sp = stg, *sq = stg + 3 * nb, *sv = stg + 7 * nb, *so = stg + 10 * nb;
  if (set) {
    const float *p = ipos, *q = iquat, *v = ivel, *o = iom;
    if (!device) {
      if (ipos) { CUDA_TRY(c, cudaMemcpyAsync(sp, ipos, sizeof(float) * 3 * nb, cudaMemcpyHostToDevice, st)); p = sp; }
      if (iquat) { CUDA_TRY(c, cudaMemcpyAsync(sq, iquat, sizeof(float) * 4 * nb, cudaMemcpyHostToDevice, st)); q = sq; }
      if (ivel) { CUDA_TRY(c, cudaMemcpyAsync(sv, ivel, sizeof(float) * 3 * nb, cudaMemcpyHostToDevice, st)); v = sv; }
      if (iom) { CUDA_TRY(c, cudaMemcpyAsync(so, iom, sizeof(float) * 3 * nb, cudaMemcpyHostToDevice, st)); o = so; }
    }
    if (c->cfg.precision == NSN_FP64)
      k_scatter_state<double><<<cdiv(nb, 128), 128, 0, st>>>(c->d64, c->d_bmap, nb, p, q, v, o);
    else
      k_scatter_state<float><<<cdiv(nb, 128), 128, 0, st>>>(c->d32, c->d_bmap, nb, p, q, v, o);
    CUDA_TRY(c, cudaGetLastError());
    if (!device) CUDA_TRY(c, cudaStreamSynchronize(st));
  } else {
    float *p = device ? opos : (opos ? sp : nullptr), *q = device ? oquat : (oquat ? sq : nullptr);
    float *v = device ? ovel : (ovel ? sv : nullptr), *o = device ? oom : (oom ? so : nullptr);
    if (c->cfg.precision == NSN_FP64)
      k_gather_state<double><<<cdiv(nb, 128), 128, 0, st>>>(c->d64, c->d_bmap, nb, p, q, v, o);
    else
      k_gather_state<float><<<cdiv(nb, 128), 128, 0, st>>>(c->d32, c->d_bmap, nb, p, q, v, o);
    CUDA_TRY(c, cudaGetLastError());
    if (!device) {
      if (opos) CUDA_TRY(c, cudaMemcpyAsync(opos, sp, sizeof(float) * 3 * nb, cudaMemcpyDeviceToHost, st));
      if (oquat) CUDA_TRY(c, cudaMemcpyAsync(oquat, sq, sizeof(float) * 4 * nb, cudaMemcpyDeviceToHost, st));
      if (ovel) CUDA_TRY(c, cudaMemcpyAsync(ovel, sv, sizeof(float) * 3 * nb, cudaMemcpyDeviceToHost, st));
      if (oom) CUDA_TRY(c, cudaMemcpyAsync(oom, so, sizeof(float) * 3 * nb, cudaMemcpyDeviceToHost, st));
      CUDA_TRY(c, cudaStreamSynchronize(st));
    }
  }
  return NSN_OK;
}

extern "C" {

nsn_status nsn_get_state(nsn_ctx *c, float *pos, float *quat, float *vel, float *omega) {
  return state_io(c, false, false, nullptr, nullptr, nullptr, nullptr, pos, quat, vel, omega);
}
nsn_status nsn_set_state(nsn_ctx *c, const float *pos, const float *quat, const float *vel, const float *omega) {
  return state_io(c, true, false, pos, quat, vel, omega, nullptr, nullptr, nullptr, nullptr);
}
nsn_status nsn_set_state_device(nsn_ctx *c, const float *pos, const float *quat, const float *vel, const float *omega) {
  return state_io(c, true, true, pos, quat, vel, omega, nullptr, nullptr, nullptr, nullptr);
}
nsn_status nsn_get_state_device(nsn_ctx *c, float *pos, float *quat, float *vel, float *omega) {
  return state_io(c, false, true, nullptr, nullptr, nullptr, nullptr, pos, quat, vel, omega);
}

nsn_status nsn_get_state_f64(nsn_ctx *c, double *pos, double *quat, double *vel, double *omega) {
  if (!c) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  const int nb = int(c->scene.kind.size());
  if (!nb) return NSN_OK;
  cudaStream_t st = c->stream;
  double *tmp;
  CUDA_TRY(c, cudaMallocAsync(&tmp, sizeof(double) * 13 * nb, st));
  double *p = pos ? tmp : nullptr, *q = quat ? tmp + 3 * nb : nullptr, *v = vel ? tmp + 7 * nb : nullptr,
         *o = omega ? tmp + 10 * nb : nullptr;
  if (c->cfg.precision == NSN_FP64)
    k_gather_state<double, double><<<cdiv(nb, 128), 128, 0, st>>>(c->d64, c->d_bmap, nb, p, q, v, o);
  else
    k_gather_state<float, double><<<cdiv(nb, 128), 128, 0, st>>>(c->d32, c->d_bmap, nb, p, q, v, o);
  CUDA_TRY(c, cudaGetLastError());
  if (pos) CUDA_TRY(c, cudaMemcpyAsync(pos, p, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, st));
  if (quat) CUDA_TRY(c, cudaMemcpyAsync(quat, q, sizeof(double) * 4 * nb, cudaMemcpyDeviceToHost, st));
  if (vel) CUDA_TRY(c, cudaMemcpyAsync(vel, v, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, st));
  if (omega) CUDA_TRY(c, cudaMemcpyAsync(omega, o, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaFreeAsync(tmp, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  return NSN_OK;
}

nsn_status nsn_get_lambda(nsn_ctx *c, double *lambda) {
  if (!c || !lambda) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  return c->cfg.precision == NSN_FP64 ? copy_out_rows<double>(c, c->d64.lam, lambda)
                                      : copy_out_rows<float>(c, c->d32.lam, lambda);
}

nsn_status nsn_get_merit_history(nsn_ctx *c, double *out, int32_t cap, int32_t *n) {
  if (!c) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  Scalars sc;
  Scalars *src = c->cfg.precision == NSN_FP64 ? c->d64.sc : c->d32.sc;
  CUDA_TRY(c, cudaMemcpyAsync(&sc, src, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  // merit at each solved Newton iteration, then at the returned iterate
  const int solved = std::min(c->last.newton_done, 1023);
  std::vector<double> hist(sc.merit, sc.merit + solved);
  hist.push_back(sc.merit_final);
  if (n) *n = int32_t(hist.size());
  if (out)
    for (int i = 0; i < std::min<int>(cap, int(hist.size())); i++) out[i] = hist[i];
  return NSN_OK;
}

nsn_status nsn_linearize(nsn_ctx *c, int32_t n_before) {
  if (!c || n_before < 0 || n_before > 1000) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  c->lin_buf = n_before & 1;
  s = c->cfg.precision == NSN_FP64 ? do_linearize<double>(c, n_before) : do_linearize<float>(c, n_before);
  if (s == NSN_OK) c->kept_buf = c->lin_buf;
  return s;
}

nsn_status nsn_apply_operator(nsn_ctx *c, const double *x, double *y) {
  if (!c || !x || !y) return NSN_ERR_INVALID_ARG;
  if (!c->linearized || c->dirty) return fail(c, NSN_ERR_BAD_STATE, "call nsn_linearize first");
  return c->cfg.precision == NSN_FP64 ? do_apply<double>(c, x, y) : do_apply<float>(c, x, y);
}

nsn_status nsn_solve(nsn_ctx *c, int32_t iters, double *dlambda, double *du) {
  if (!c || iters < 0) return NSN_ERR_INVALID_ARG;
  if (!c->linearized || c->dirty) return fail(c, NSN_ERR_BAD_STATE, "call nsn_linearize first");
  return c->cfg.precision == NSN_FP64 ? do_solve<double>(c, iters, dlambda, du) : do_solve<float>(c, iters, dlambda, du);
}

nsn_status nsn_get_system(nsn_ctx *c, double *b, double *diag, double *hvec, double *g) {
  if (!c) return NSN_ERR_INVALID_ARG;
  if (!c->linearized || c->dirty) return fail(c, NSN_ERR_BAD_STATE, "call nsn_linearize first");
  return c->cfg.precision == NSN_FP64 ? do_system<double>(c, b, diag, hvec, g) : do_system<float>(c, b, diag, hvec, g);
}

nsn_status nsn_time_operator(nsn_ctx *c, int32_t iters, float *ms_body_pass, float *ms_row_pass) {
  if (!c || iters <= 0) return NSN_ERR_INVALID_ARG;
  if (c->dirty) return fail(c, NSN_ERR_BAD_STATE, "call nsn_step first");
  return c->cfg.precision == NSN_FP64 ? do_time_operator<double>(c, iters, ms_body_pass, ms_row_pass)
                                      : do_time_operator<float>(c, iters, ms_body_pass, ms_row_pass);
}

nsn_status nsn_operator_sizes(nsn_ctx *c, int64_t *sizes) {
  if (!c || !sizes) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  const Layout &L = c->L;
  sizes[0] = L.nr; sizes[1] = L.np; sizes[2] = L.R; sizes[3] = L.Rpair; sizes[4] = L.nt;
  sizes[5] = L.ER; sizes[6] = L.EV; sizes[7] = (int64_t)c->dbytes;
  return NSN_OK;
}

nsn_status nsn_set_warm_start(nsn_ctx *c, int32_t mode) {
  if (!c) return NSN_ERR_INVALID_ARG;
  const int base = mode & 0xff, fric = (mode & NSN_WARM_FRICTION) ? 1 : 0, pre = (mode & NSN_WARM_PRECOND) ? 1 : 0;
  if (base < NSN_WARM_ZERO || base > NSN_WARM_LEARNED || (mode & ~(0xff | NSN_WARM_FRICTION | NSN_WARM_PRECOND)))
    return NSN_ERR_INVALID_ARG;
  if ((base != c->warm_mode || fric != c->warm_friction || pre != c->warm_precond) && c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->warm_mode = base;
  c->warm_friction = fric;
  c->warm_precond = pre;
  return NSN_OK;
}

nsn_status nsn_islands(nsn_ctx *c, int32_t *n_islands, int32_t *body_island) {
  if (!c || !n_islands) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  *n_islands = c->L.ni;
  if (body_island) std::copy(c->L.body_isl.begin(), c->L.body_isl.end(), body_island);
  return NSN_OK;
}

nsn_status nsn_island_stats(nsn_ctx *c, int32_t cap, double *merit0, double *merit_final, int32_t *stopped_at) {
  if (!c) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  const int ni = c->L.ni;
  if (cap < ni) return fail(c, NSN_ERR_INVALID_ARG, "nsn_island_stats: cap %d < %d islands", cap, ni);
  if (!ni) return NSN_OK;
  const bool f64 = c->cfg.precision == NSN_FP64;
  const IslState &I = f64 ? c->d64.isl : c->d32.isl;
  cudaStream_t st = c->stream;
  if (merit0) CUDA_TRY(c, cudaMemcpyAsync(merit0, I.m0, sizeof(double) * ni, cudaMemcpyDeviceToHost, st));
  if (merit_final) CUDA_TRY(c, cudaMemcpyAsync(merit_final, I.mf, sizeof(double) * ni, cudaMemcpyDeviceToHost, st));
  if (stopped_at) CUDA_TRY(c, cudaMemcpyAsync(stopped_at, I.stop, sizeof(int32_t) * ni, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  return NSN_OK;
}

nsn_status nsn_island_stop_copy(nsn_ctx *c, int32_t *dst_device) {
  if (!c || !dst_device) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  if (!c->L.ni) return NSN_OK;
  const int *src = c->cfg.precision == NSN_FP64 ? c->d64.isl.stop : c->d32.isl.stop;
  CUDA_TRY(c, cudaMemcpyAsync(dst_device, src, sizeof(int32_t) * c->L.ni, cudaMemcpyDeviceToDevice, c->stream));
  return NSN_OK;
}

}  // extern "C"

namespace {
// v += h g: the unconstrained velocity the collider predicts with (Sec. 10)
__global__ void k_add_gravity(float *vel, int nb, float gx, float gy, float gz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  vel[3 * i] += gx; vel[3 * i + 1] += gy; vel[3 * i + 2] += gz;
}

nsn_status collide_once(nsn_ctx *c, nsn_collider *col) {
  const int nb = int(c->scene.kind.size());
  double t0 = now_ms();
  int32_t info[4];
  nsn_status s = nsn_collider_info(col, info);
  if (s != NSN_OK) return fail(c, s, "nsn_collide_and_step: bad collider");
  if (info[0] != nb) return fail(c, NSN_ERR_INVALID_ARG, "nsn_collide_and_step: the collider has %d bodies, the scene %d", info[0], nb);
  if ((s = ensure_built(c)) != NSN_OK) return s;
  cudaStream_t st = c->stream;
  if (c->col_state_nb != nb) {
    if (c->col_state) cudaFree(c->col_state);
    c->col_state = nullptr;
    c->col_state_nb = 0;
    CUDA_TRY(c, cudaMalloc(&c->col_state, sizeof(float) * 13 * std::max(nb, 1)));
    c->col_state_nb = nb;
  }
  if (!c->col_found) {
    CUDA_TRY(c, cudaMalloc(&c->col_found, sizeof(int32_t)));
    CUDA_TRY(c, cudaMallocHost(&c->col_found_h, sizeof(int32_t)));
  }
  float *pos = c->col_state, *quat = pos + 3 * size_t(nb), *vel = pos + 7 * size_t(nb), *om = pos + 10 * size_t(nb);
  if ((s = state_io(c, false, true, nullptr, nullptr, nullptr, nullptr, pos, quat, vel, om)) != NSN_OK) return s;
  const float h = float(c->cfg.h);
  if (nb) k_add_gravity<<<cdiv(nb, 256), 256, 0, st>>>(vel, nb, h * float(c->cfg.gravity[0]), h * float(c->cfg.gravity[1]),
                                                       h * float(c->cfg.gravity[2]));
  CUDA_TRY(c, cudaGetLastError());
  // the collider works on its own stream: the state export must be complete
  CUDA_TRY(c, cudaStreamSynchronize(st));
  cudaStream_t cs = nsn_collider_stream_of(col);
  for (int attempt = 0; attempt < 2; attempt++) {
    if (c->col_cap == 0) {
      const int cap = std::max(1024, int(c->scene.contacts.size()) + int(c->scene.contacts.size()) / 4);
      CUDA_TRY(c, cudaMalloc(&c->col_body, sizeof(int32_t) * 2 * size_t(cap)));
      CUDA_TRY(c, cudaMalloc(&c->col_f, sizeof(float) * 11 * size_t(cap)));
      CUDA_TRY(c, cudaMallocHost(&c->col_body_h, sizeof(int32_t) * 2 * size_t(cap)));
      CUDA_TRY(c, cudaMallocHost(&c->col_f_h, sizeof(float) * 11 * size_t(cap)));
      c->col_cap = cap;
    }
    const size_t cap = size_t(c->col_cap);
    float *pa = c->col_f, *pb = pa + 3 * cap, *n = pa + 6 * cap, *d = pa + 9 * cap, *mu = pa + 10 * cap;
    s = nsn_collider_run_async(col, pos, quat, vel, om, c->col_cap, c->col_body, pa, pb, n, d, mu, c->col_found);
    if (s != NSN_OK) return fail(c, s, "nsn_collide_and_step: %s", nsn_collider_last_error(col));
    CUDA_TRY(c, cudaMemcpyAsync(c->col_found_h, c->col_found, sizeof(int32_t), cudaMemcpyDeviceToHost, cs));
    CUDA_TRY(c, cudaStreamSynchronize(cs));
    const int found = *c->col_found_h;
    if (found > c->col_cap) {   // grow and run again
      cudaFree(c->col_body); cudaFree(c->col_f); cudaFreeHost(c->col_body_h); cudaFreeHost(c->col_f_h);
      c->col_body = nullptr; c->col_f = nullptr; c->col_body_h = nullptr; c->col_f_h = nullptr;
      c->col_cap = 0;
      const int cap2 = found + found / 4 + 1024;
      CUDA_TRY(c, cudaMalloc(&c->col_body, sizeof(int32_t) * 2 * size_t(cap2)));
      CUDA_TRY(c, cudaMalloc(&c->col_f, sizeof(float) * 11 * size_t(cap2)));
      CUDA_TRY(c, cudaMallocHost(&c->col_body_h, sizeof(int32_t) * 2 * size_t(cap2)));
      CUDA_TRY(c, cudaMallocHost(&c->col_f_h, sizeof(float) * 11 * size_t(cap2)));
      c->col_cap = cap2;
      continue;
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->col_body_h, c->col_body, sizeof(int32_t) * 2 * size_t(found), cudaMemcpyDeviceToHost, cs));
    const float *src[5] = {pa, pb, n, d, mu};
    const size_t w[5] = {3, 3, 3, 1, 1}, o[5] = {0, 3 * cap, 6 * cap, 9 * cap, 10 * cap};
    for (int k = 0; k < 5; k++)
      CUDA_TRY(c, cudaMemcpyAsync(c->col_f_h + o[k], src[k], sizeof(float) * w[k] * size_t(found), cudaMemcpyDeviceToHost, cs));
    CUDA_TRY(c, cudaStreamSynchronize(cs));
    std::vector<nsn_contact> &rec = c->col_rec;
    rec.resize(size_t(found));
    const float *hf = c->col_f_h;
    const int nth = layout_threads(found);
    parallel_for_threads(nth, [&](int h) {
      const int i0 = int((long long)found * h / nth), i1 = int((long long)found * (h + 1) / nth);
      for (int i = i0; i < i1; i++) {
        nsn_contact &r = rec[i];
        r.body_a = c->col_body_h[2 * i];
        r.body_b = c->col_body_h[2 * i + 1];
        for (int k = 0; k < 3; k++) { r.pa[k] = hf[3 * i + k]; r.pb[k] = hf[3 * cap + 3 * i + k]; r.n[k] = hf[6 * cap + 3 * i + k]; }
        r.d = hf[9 * cap + i];
        r.mu = hf[10 * cap + i];
      }
    });
    c->scene.contacts.swap(rec);
    c->dirty = true;
    c->phase_ms[NSN_PHASE_COLLIDE] = 0.0;
    phase_tick(c, NSN_PHASE_COLLIDE, t0);
    return NSN_OK;
  }
  return fail(c, NSN_ERR_OUT_OF_MEMORY, "nsn_collide_and_step: contact buffer");
}
}  // namespace

extern "C" {

nsn_status nsn_collide_and_step(nsn_ctx *c, nsn_collider *col, int32_t nsteps, nsn_stats *stats) {
  if (!c || !col || nsteps < 0) return NSN_ERR_INVALID_ARG;
  for (int k = 0; k < nsteps; k++) {
    nsn_status s = collide_once(c, col);
    if (s != NSN_OK) return s;
    if ((s = nsn_step(c, 1, stats)) != NSN_OK) return s;
  }
  return NSN_OK;
}

nsn_status nsn_best_restored(nsn_ctx *c, int32_t *n) {
  if (!c || !n) return NSN_ERR_INVALID_ARG;
  *n = c->best_restored;
  return NSN_OK;
}

nsn_status nsn_get_phase_times(nsn_ctx *c, double *ms) {
  if (!c || !ms) return NSN_ERR_INVALID_ARG;
  for (int k = 0; k < NSN_PHASES; k++) ms[k] = c->phase_ms[k];
  return NSN_OK;
}

nsn_status nsn_get_prev_lambda(nsn_ctx *c, double *lambda) {
  if (!c || !lambda) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  std::vector<double> v;
  s = c->cfg.precision == NSN_FP64 ? save_lam_prev<double>(c, v) : save_lam_prev<float>(c, v);
  if (s != NSN_OK) return s;
  if (v.empty()) v.assign(c->L.R, 0.0);
  std::copy(v.begin(), v.end(), lambda);
  return NSN_OK;
}

nsn_status nsn_record_decisions(nsn_ctx *c, int32_t iters) {
  if (!c || iters < 0 || iters > 100000) return NSN_ERR_INVALID_ARG;
  c->dlog_iters = iters;
  return NSN_OK;
}

nsn_status nsn_get_decisions(nsn_ctx *c, uint8_t *rows, uint8_t *islands, uint16_t *cr) {
  if (!c) return NSN_ERR_INVALID_ARG;
  if (c->dlog_iters <= 0 || !c->dlog_buf || c->dirty)
    return fail(c, NSN_ERR_BAD_STATE, "nsn_get_decisions: no logged step (nsn_record_decisions, then nsn_step)");
  const Layout &L = c->L;
  const int it = c->dlog_iters, R = L.R, ni = L.ni;
  std::vector<uint8_t> h(size_t(it) * (size_t(R) + 3 * size_t(ni)));
  CUDA_TRY(c, cudaMemcpyAsync(h.data(), c->dlog_buf, h.size(), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const size_t o_rows = 2 * size_t(it) * ni, o_isl = o_rows + size_t(it) * R;
  if (cr) std::memcpy(cr, h.data(), 2 * size_t(it) * ni);
  if (rows)
    for (int n = 0; n < it; n++)
      for (int i = 0; i < R; i++) rows[size_t(n) * R + L.row_abi[i]] = h[o_rows + size_t(n) * R + i];
  if (islands) std::copy(h.begin() + o_isl, h.end(), islands);
  return NSN_OK;
}

nsn_status nsn_island_stop_device(nsn_ctx *c, const int32_t **stopped_at) {
  if (!c || !stopped_at) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  *stopped_at = c->cfg.precision == NSN_FP64 ? c->d64.isl.stop : c->d32.isl.stop;
  return NSN_OK;
}

nsn_status nsn_clear_warm_start(nsn_ctx *c) {
  if (!c) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  if (!c->L.R) return NSN_OK;
  if (c->cfg.precision == NSN_FP64) CUDA_TRY(c, cudaMemsetAsync(c->d64.lam_prev, 0, sizeof(double) * c->L.R, c->stream));
  else CUDA_TRY(c, cudaMemsetAsync(c->d32.lam_prev, 0, sizeof(float) * c->L.R, c->stream));
  return NSN_OK;
}

nsn_status nsn_get_warm_stats(nsn_ctx *c, double *merit_zero, double *merit_warm, int32_t *rejected) {
  if (!c) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  Scalars sc;
  Scalars *src = c->cfg.precision == NSN_FP64 ? c->d64.sc : c->d32.sc;
  CUDA_TRY(c, cudaMemcpyAsync(&sc, src, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (merit_zero) *merit_zero = sc.merit0;
  if (merit_warm) *merit_warm = c->warm_mode == NSN_WARM_LEARNED ? sc.merit_warm2 : sc.merit_warm;
  if (rejected) *rejected = sc.warm_rejected;
  return NSN_OK;
}

nsn_status nsn_mlp_set_params(nsn_ctx *c, const float *params, int32_t n) {
  if (!c || !params || n != mlp::NPARAM) return NSN_ERR_INVALID_ARG;
  MlpState &m = c->mlp;
  nsn_status s;
  if (!m.pf) {
    if ((s = dalloc(c, &m.pf, mlp::NPARAM)) || (s = dalloc(c, &m.gr, mlp::NPARAM)) || (s = dalloc(c, &m.m, mlp::NPARAM)) ||
        (s = dalloc(c, &m.v, mlp::NPARAM)) || (s = dalloc(c, &m.pb, mlp::NPARAM)) || (s = dalloc(c, &m.err, 1)))
      return s;
    CUDA_TRY(c, cudaMemsetAsync(m.err, 0, sizeof(int), c->stream));
  }
  CUDA_TRY(c, cudaMemcpyAsync(m.pf, params, sizeof(float) * n, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(m.m, 0, sizeof(float) * n, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(m.v, 0, sizeof(float) * n, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(m.gr, 0, sizeof(float) * n, c->stream));
  mlp::k_to_bf16<<<cdiv(n, 256), 256, 0, c->stream>>>(m.pf, m.pb, n);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  m.adam_t = 0;
  m.ready = true;
  return NSN_OK;
}

nsn_status nsn_mlp_get_params(nsn_ctx *c, float *params, float *grads, int32_t n) {
  if (!c || n != mlp::NPARAM || !c->mlp.ready) return NSN_ERR_INVALID_ARG;
  if (params) CUDA_TRY(c, cudaMemcpyAsync(params, c->mlp.pf, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
  if (grads) CUDA_TRY(c, cudaMemcpyAsync(grads, c->mlp.gr, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return NSN_OK;
}

nsn_status nsn_mlp_forward(nsn_ctx *c, const float *X, int32_t n, float *Y) {
  if (!c || !X || !Y || n < 0 || !c->mlp.ready) return NSN_ERR_INVALID_ARG;
  nsn_status s = mlp_workspace(c, kMlpChunk);
  if (s != NSN_OK) return s;
  mlp_infer(c, X, n, Y, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  return mlp_check(c, c->stream);
}

nsn_status nsn_mlp_time_forward(nsn_ctx *c, const float *X, int32_t n, float *Y, int32_t reps, float *ms) {
  if (!c || !X || !Y || !ms || n < 0 || reps < 1 || !c->mlp.ready) return NSN_ERR_INVALID_ARG;
  nsn_status s = mlp_workspace(c, kMlpChunk);
  if (s != NSN_OK) return s;
  if (!c->ev0) CUDA_TRY(c, cudaEventCreate(&c->ev0));
  if (!c->ev1) CUDA_TRY(c, cudaEventCreate(&c->ev1));
  CUDA_TRY(c, cudaEventRecord(c->ev0, c->stream));
  for (int k = 0; k < reps; k++) mlp_infer(c, X, n, Y, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaEventRecord(c->ev1, c->stream));
  CUDA_TRY(c, cudaEventSynchronize(c->ev1));
  float t = 0.f;
  CUDA_TRY(c, cudaEventElapsedTime(&t, c->ev0, c->ev1));
  *ms = t / float(reps);
  return mlp_check(c, c->stream);
}

nsn_status nsn_mlp_train_step(nsn_ctx *c, const float *X, const float *T, const float *w, int32_t n, float lr, float *loss) {
  if (!c || !X || !T || !w || n <= 0 || !c->mlp.ready) return NSN_ERR_INVALID_ARG;
  return mlp_train(c, X, T, w, n, lr, loss);
}

nsn_status nsn_contact_features(nsn_ctx *c, float *X, float *Ytarget) {
  if (!c) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  return c->cfg.precision == NSN_FP64 ? do_features<double>(c, X, Ytarget) : do_features<float>(c, X, Ytarget);
}

nsn_status nsn_tuning(nsn_ctx *c, int32_t *body_lanes, float *ms3) {
  if (!c) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  if (body_lanes) *body_lanes = c->cfg.precision == NSN_FP64 ? c->d64.G : c->d32.G;
  if (ms3) for (int k = 0; k < 3; k++) ms3[k] = c->tune_ms[k];
  return NSN_OK;
}

nsn_status nsn_resident_info(nsn_ctx *c, int32_t *info6) {
  if (!c || !info6) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  const bool f64 = c->cfg.precision == NSN_FP64;
  const int on = f64 ? c->d64.res_on : c->d32.res_on;
  info6[0] = on ? c->L.n_res : 0;
  info6[1] = on ? int(c->L.gres.size() / 10) : 0;
  info6[2] = on ? c->L.res_rows : 0;
  info6[3] = on ? c->L.res_ent : 0;
  info6[4] = on ? (f64 ? c->d64.res_smem : c->d32.res_smem) : 0;
  info6[5] = on ? (f64 ? c->d64.nblk_res : c->d32.nblk_res) : 0;
  return NSN_OK;
}

nsn_status nsn_time_resident(nsn_ctx *c, int32_t iters, float *ms, double *work4) {
  if (!c || iters < 1) return NSN_ERR_INVALID_ARG;
  nsn_status s = ensure_built(c);
  if (s != NSN_OK) return s;
  s = c->cfg.precision == NSN_FP64 ? do_time_resident<double>(c, iters, ms, work4)
                                   : do_time_resident<float>(c, iters, ms, work4);
  if (s == NSN_ERR_INVALID_ARG) c->err = "nsn_time_resident: no island-resident CR in this context";
  return s;
}

nsn_status nsn_set_body_lanes(nsn_ctx *c, int32_t lanes) {
  if (!c || (lanes != 0 && lanes != 4 && lanes != 8 && lanes != 16)) return NSN_ERR_INVALID_ARG;
  if (lanes != c->forced_lanes) {
    c->forced_lanes = lanes;
    c->tuned_lanes = 0;   // lanes = 0: tune again
    c->dirty = true;      // rebuilt (state kept) before the next use
  }
  return NSN_OK;
}

nsn_status nsn_last_launch_count(nsn_ctx *c, int32_t *kernels_per_step) {
  if (!c || !kernels_per_step) return NSN_ERR_INVALID_ARG;
  *kernels_per_step = c->launches_per_step;
  return NSN_OK;
}

}  // extern "C"

// =====================================================================================
// Allocation-free operator apply.
//
// Some callers cannot allocate device memory at the point where they need an
// operator product: a host application that owns the device's memory and hands
// the library a fixed budget with nothing to spare, and a real-time control
// loop that must not block in the device allocator (cudaMalloc can synchronise
// the device and take milliseconds).  For them nsn_apply_operator_noalloc
// computes y = (J H~^-1 J^T + C + eps I) x with the same two kernels as the CR
// loop, but keeps the per-entry scratch, the per-block partials and the flags
// in the file-scope device arrays below (part of the library image, resident
// on every device that loads it until the process exits) instead of in memory
// allocated by the context.

namespace {

constexpr int kNoallocMaxEntries = NSN_NOALLOC_MAX_ENTRIES;
constexpr int kNoallocMaxRows = NSN_NOALLOC_MAX_ENTRIES / 2;  // a row has at least 2 slots
constexpr int kNoallocMaxBlocks = 8192;                        // grid cap the partials can hold
static __device__ __align__(256) float g_noalloc_t[kNoallocMaxEntries];
// x and y in the context's internal (island) row order
static __device__ __align__(256) float g_noalloc_x[kNoallocMaxRows];
static __device__ __align__(256) float g_noalloc_y[kNoallocMaxRows];
static __device__ __align__(256) DS g_noalloc_part[2 * kNoallocMaxBlocks * NPART];
static __device__ __align__(256) Flags g_noalloc_flags;  // never written by the apply kernels

struct NoallocPtrs {
  float *t = nullptr, *x = nullptr, *y = nullptr;
  DS *part = nullptr;
  Flags *flags = nullptr;
  CUcontext ctx = nullptr;   // the CUDA context the addresses belong to
  bool ready = false;
};
constexpr int kMaxDevices = 64;
// Resolved addresses per device.  Contexts on different host threads may make
// their first call at the same time: the table is read and written only under
// g_noalloc_mu, and each call takes a copy of its entry.
std::mutex g_noalloc_mu;
NoallocPtrs g_noalloc_dev[kMaxDevices];

// cuCtxGetCurrent, obtained through the runtime (no link against the driver library)
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
CtxGetCurrentFn ctx_get_current() {
  static const CtxGetCurrentFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(p);
  }();
  return fn;
}

// Host code cannot use the arrays' names as device addresses: they are
// host-side stand-ins.  Resolve them once per device, with that device
// current, and again if the device's context changed since (after
// cudaDeviceReset the module is loaded anew and the arrays may move).
nsn_status noalloc_setup(nsn_ctx *c, NoallocPtrs *out) {
  int dev = 0;
  CUDA_TRY(c, cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(c, NSN_ERR_INVALID_ARG, "device index %d out of range", dev);
  CUcontext cur = nullptr;
  const CtxGetCurrentFn get = ctx_get_current();
  if (!get || get(&cur) != CUDA_SUCCESS)
    return fail(c, NSN_ERR_CUDA, "nsn_apply_operator_noalloc: cuCtxGetCurrent unavailable");
  if (!cur) {   // first runtime call of this host thread: bind the device's primary context
    CUDA_TRY(c, cudaSetDevice(dev));
    if (get(&cur) != CUDA_SUCCESS || !cur)
      return fail(c, NSN_ERR_CUDA, "nsn_apply_operator_noalloc: no current CUDA context");
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoallocPtrs &p = g_noalloc_dev[dev];
  if (!p.ready || p.ctx != cur) {
    p.ready = false;
    void *t = nullptr, *part = nullptr, *fl = nullptr, *x = nullptr, *y = nullptr;
    const cudaError_t e[5] = {cudaGetSymbolAddress(&t, g_noalloc_t), cudaGetSymbolAddress(&part, g_noalloc_part),
                              cudaGetSymbolAddress(&fl, g_noalloc_flags), cudaGetSymbolAddress(&x, g_noalloc_x),
                              cudaGetSymbolAddress(&y, g_noalloc_y)};
    for (cudaError_t ei : e)
      if (ei != cudaSuccess) return fail(c, NSN_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(ei));
    p.t = static_cast<float *>(t);
    p.x = static_cast<float *>(x);
    p.y = static_cast<float *>(y);
    p.part = static_cast<DS *>(part);
    p.flags = static_cast<Flags *>(fl);
    p.ctx = cur;
    p.ready = true;
  }
  *out = p;
  return NSN_OK;
}

// y[row_abi[i]] = x[i] (scatter) or y[i] = x[row_abi[i]] (gather)
__global__ void k_permute_rows(float *dst, const float *src, const int *row_abi, int n, int scatter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (scatter) dst[row_abi[i]] = src[i];
  else dst[i] = src[row_abi[i]];
}

}  // namespace

extern "C" nsn_status nsn_apply_operator_noalloc(nsn_ctx *c, const float *x, float *y, void *stream) {
  if (!c || !x || !y) return NSN_ERR_INVALID_ARG;
  if (c->cfg.precision != NSN_FP32) return fail(c, NSN_ERR_INVALID_ARG, "nsn_apply_operator_noalloc needs an FP32 context");
  if (c->dirty || c->kept_buf < 0) return fail(c, NSN_ERR_BAD_STATE, "no kept system: call nsn_step or nsn_linearize first");
  const Layout &L = c->L;
  const size_t nslots = size_t(2) * L.Rpair + size_t(12) * L.nt;
  if (nslots > size_t(kNoallocMaxEntries))
    return fail(c, NSN_ERR_INVALID_ARG,
                "nsn_apply_operator_noalloc: %lld row slots (2 per contact or joint row, 4 per tet row) exceed the "
                "static scratch of %d",
                (long long)nslots, kNoallocMaxEntries);
  if (c->d32.max_blk > kNoallocMaxBlocks)
    return fail(c, NSN_ERR_INVALID_ARG, "nsn_apply_operator_noalloc: %d blocks per grid exceed the static partials of %d",
                c->d32.max_blk, kNoallocMaxBlocks);
  NoallocPtrs npv;
  nsn_status s = noalloc_setup(c, &npv);
  if (s != NSN_OK) return s;
  const NoallocPtrs *np = &npv;
  if (L.R == 0) return NSN_OK;
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : c->stream;
  Dev<float> D = c->d32;
  D.t = np->t;
  D.part_row = np->part;
  D.fl = np->flags;
  D.z = np->x;
  D.Az = np->y;
  D.isl_on = 0;  // every row takes part
  // world-side slots are read but never written: clear the shared scratch
  CUDA_TRY(c, cudaMemsetAsync(np->t, 0, sizeof(float) * nslots, st));
  k_permute_rows<<<cdiv(L.R, 256), 256, 0, st>>>(np->x, x, D.row_abi_dev, L.R, 0);
  const int nb = D.nblk_body_r + D.nblk_body_p, nrw = D.nblk_row_pair + D.nblk_row_tet;
  if (nb) {
    if (D.G == 4) k_body_pass<float, 4, BM_APPLY><<<nb, BLOCK, 0, st>>>(D, np->x, c->kept_buf, 0, 1);
    else if (D.G == 16) k_body_pass<float, 16, BM_APPLY><<<nb, BLOCK, 0, st>>>(D, np->x, c->kept_buf, 0, 1);
    else k_body_pass<float, 8, BM_APPLY><<<nb, BLOCK, 0, st>>>(D, np->x, c->kept_buf, 0, 1);
  }
  k_row_pass<float, RM_APPLY><<<nrw, BLOCK, 0, st>>>(D, 1);
  k_permute_rows<<<cdiv(L.R, 256), 256, 0, st>>>(y, np->y, D.row_abi_dev, L.R, 1);
  CUDA_TRY(c, cudaGetLastError());
  return NSN_OK;
}
