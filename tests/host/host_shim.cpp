// Host-only test harness around the library's set-up code (setup.cpp): the
// box decomposition, DoF classes, partition of unity, nodal loads, 3-2-1 pins,
// wave grouping and the static tile-task schedules of the layer-block
// factorisation and block triangular solves.  Test infrastructure: compiled
// with the host compiler together with setup.cpp (no CUDA calls), loaded only
// by tests/.
//
// Schedules are checked two ways:
//  * race check: the memory footprint (read and written byte ranges) of every
//    task; two tasks of one step (one launch, CTAs in any order) or of two
//    stream groups (no ordering at all) must not touch a byte that one of them
//    writes;
//  * host execution: every task run in plain loops with the semantics of the
//    tile kernels (k_tile_task, k_solve_step and its variants), groups
//    interleaved at random and the tasks of a step in random order.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "internal.h"

namespace {

struct HostCheck {
  msgfem h;
  msgfem_status st = MSGFEM_OK;
  std::vector<char> pool_mem;
  char* pool = nullptr;
  int wave = -1;
  WaveSched* w = nullptr;
  // coarse schedules
  int coarse = 0;
  std::vector<double> cscr, cid;   // scratch and identity strip of the split coarse inverse
};

struct Iv {
  uintptr_t lo, hi;
  int task, group;
  bool wr;
};

template <typename T>
void rows(std::vector<Iv>& out, const void* p, int nrows, int ld, int ncols, bool wr, int task, int group) {
  if (p == nullptr || nrows <= 0 || ncols <= 0) return;
  const T* b = static_cast<const T*>(p);
  if (ld == ncols) {
    out.push_back({(uintptr_t)b, (uintptr_t)(b + (size_t)nrows * ld), task, group, wr});
    return;
  }
  for (int r = 0; r < nrows; ++r)
    out.push_back({(uintptr_t)(b + (size_t)r * ld), (uintptr_t)(b + (size_t)r * ld + ncols), task, group, wr});
}

template <typename T>
void footprint(const TileTaskT<T>& t, std::vector<Iv>& out, int id, int g) {
  if (t.flags & G_POTRF) {
    rows<T>(out, t.C, 64, t.ldc, 64, true, id, g);
    rows<T>(out, t.P, 64, t.ldc, 64, true, id, g);
    return;
  }
  rows<T>(out, t.A, 64, t.lda, t.K, false, id, g);
  if (t.flags & G_TRANSB)
    rows<T>(out, t.B, 64, t.ldb, t.K, false, id, g);
  else
    rows<T>(out, t.B, t.K, t.ldb, 64, false, id, g);
  if (t.flags & G_POSTMUL) rows<T>(out, t.P, 64, t.ldc, 64, false, id, g);
  rows<T>(out, t.C, 64, t.ldc, 64, true, id, g);
}

// full-layout multivectors gathered from / scattered to, per subdomain
struct MvArgs {
  double* const* src = nullptr;
  double* const* dst = nullptr;
  int gather_neg = 0, scatter_add = 0;
};

template <typename T>
void footprint(const SolveTaskT<T>& t, int pc, const MvArgs& mv, std::vector<Iv>& out, int id, int g) {
  if (t.K > 0) {
    if (t.flags & S_TRANSA)
      rows<T>(out, t.A, t.K, t.lda, 64, false, id, g);
    else
      rows<T>(out, t.A, 64, t.lda, t.K, false, id, g);
    rows<T>(out, t.B, t.K, pc, pc, false, id, g);
  }
  if (t.flags & S_INIT_TILE) rows<T>(out, t.init, 64, pc, pc, false, id, g);
  rows<T>(out, t.C, 64, pc, pc, true, id, g);
  for (int r = 0; r < 64; ++r) {
    if ((t.flags & S_INIT_GATHER) && t.gmap[r] >= 0)
      rows<double>(out, mv.src[t.sub] + ((size_t)t.row_off + t.gmap[r]) * pc, 1, pc, pc, false, id, g);
    if ((t.flags & S_SCATTER) && t.smap[r] >= 0)
      rows<double>(out, mv.dst[t.sub] + ((size_t)t.row_off + t.smap[r]) * pc, 1, pc, pc, true, id, g);
  }
}

// Conflicting pairs among the intervals: overlapping byte ranges of two
// different tasks, at least one written (cross_group_only: the two tasks must
// also be in different stream groups).  The first one found is described in
// *first.
long long conflicts(std::vector<Iv>& iv, bool cross_group_only, std::string* first) {
  std::sort(iv.begin(), iv.end(), [](const Iv& a, const Iv& b) { return a.lo < b.lo; });
  std::vector<const Iv*> open;
  long long n = 0;
  for (const Iv& x : iv) {
    size_t k = 0;
    for (size_t i = 0; i < open.size(); ++i)
      if (open[i]->hi > x.lo) open[k++] = open[i];
    open.resize(k);
    for (const Iv* y : open) {
      if (y->task == x.task || !(x.wr || y->wr)) continue;
      if (cross_group_only && y->group == x.group) continue;
      if (first != nullptr && first->empty()) {
        char buf[160];
        snprintf(buf, sizeof buf, "tasks %d (group %d) and %d (group %d) overlap at byte offset %lld", y->task,
                 y->group, x.task, x.group, (long long)(x.lo - y->lo));
        *first = buf;
      }
      ++n;
    }
    open.push_back(&x);
  }
  return n;
}

template <typename Task, typename FP>
long long race_check(const std::vector<std::vector<SchedStep>>& steps, const std::vector<Task>& tasks, FP fp,
                     std::string* first) {
  long long n = 0;
  std::vector<Iv> all;
  for (size_t g = 0; g < steps.size(); ++g)
    for (const SchedStep& st : steps[g]) {
      std::vector<Iv> iv;
      for (int i = st.first; i < st.first + st.count; ++i) fp(tasks[i], iv, i, (int)g);
      all.insert(all.end(), iv.begin(), iv.end());
      n += conflicts(iv, false, first);
    }
  n += conflicts(all, true, first);
  return n;
}

// ---- host execution with the kernels' semantics ---------------------------

template <typename T>
void exec(const TileTaskT<T>& t, int* notspd) {
  if (t.flags & G_POTRF) {
    static thread_local double A[64][64], X[64][64];
    for (int r = 0; r < 64; ++r)
      for (int c = 0; c < 64; ++c) A[r][c] = c <= r ? (double)t.C[(size_t)r * t.ldc + c] : 0.0;
    bool bad = false;
    for (int j = 0; j < 64; ++j) {
      double d = A[j][j];
      for (int m = 0; m < j; ++m) d -= A[j][m] * A[j][m];
      if (!(d > 0.0)) { bad = true; d = 1e-300; }
      A[j][j] = std::sqrt(d);
      for (int i = j + 1; i < 64; ++i) {
        double v = A[i][j];
        for (int m = 0; m < j; ++m) v -= A[i][m] * A[j][m];
        A[i][j] = v / A[j][j];
      }
    }
    for (int c = 0; c < 64; ++c)
      for (int i = 0; i < 64; ++i) {
        if (i < c) { X[i][c] = 0.0; continue; }
        if (i == c) { X[i][c] = 1.0 / A[i][i]; continue; }
        double v = 0.0;
        for (int m = c; m < i; ++m) v += A[i][m] * X[m][c];
        X[i][c] = -v / A[i][i];
      }
    T* Li = const_cast<T*>(t.P);
    for (int r = 0; r < 64; ++r)
      for (int c = 0; c < 64; ++c) {
        t.C[(size_t)r * t.ldc + c] = (T)(c <= r ? A[r][c] : 0.0);
        Li[(size_t)r * t.ldc + c] = (T)(c <= r ? X[r][c] : 0.0);
      }
    if (bad && notspd) ++*notspd;
    return;
  }
  static thread_local double acc[64][64], tmp[64][64];
  const bool tb = (t.flags & G_TRANSB) != 0;
  for (int r = 0; r < 64; ++r)
    for (int c = 0; c < 64; ++c) {
      double v = 0.0;
      for (int k = 0; k < t.K; ++k)
        v += (double)t.A[(size_t)r * t.lda + k] * (double)(tb ? t.B[(size_t)c * t.ldb + k] : t.B[(size_t)k * t.ldb + c]);
      acc[r][c] = v;
    }
  if (t.flags & G_POSTMUL) {
    for (int r = 0; r < 64; ++r)
      for (int c = 0; c < 64; ++c) {
        double v = 0.0;
        for (int m = 0; m < 64; ++m) v += (double)t.P[(size_t)r * t.ldc + m] * acc[m][c];
        tmp[r][c] = v;
      }
    memcpy(acc, tmp, sizeof acc);
  }
  const double sg = (t.flags & G_NEG) ? -1.0 : 1.0;
  for (int r = 0; r < 64; ++r)
    for (int c = 0; c < 64; ++c) {
      T* p = t.C + (size_t)r * t.ldc + c;
      const T v = (T)(sg * acc[r][c]);
      *p = (t.flags & G_ACC) ? (T)(*p + v) : v;
    }
}

template <typename T>
void exec(const SolveTaskT<T>& t, int pc, const MvArgs& mv) {
  const bool ta = (t.flags & S_TRANSA) != 0;
  const double sg = (t.flags & S_NEG) ? -1.0 : 1.0;
  const double gs = mv.gather_neg ? -1.0 : 1.0;
  const double* gfull = (t.flags & S_INIT_GATHER) ? mv.src[t.sub] + (size_t)t.row_off * pc : nullptr;
  double* sfull = (t.flags & S_SCATTER) ? mv.dst[t.sub] + (size_t)t.row_off * pc : nullptr;
  std::vector<double> out((size_t)64 * pc);
  for (int r = 0; r < 64; ++r)
    for (int c = 0; c < pc; ++c) {
      double v = 0.0;
      for (int k = 0; k < t.K; ++k)
        v += (double)(ta ? t.A[(size_t)k * t.lda + r] : t.A[(size_t)r * t.lda + k]) * (double)t.B[(size_t)k * pc + c];
      v *= sg;
      if (t.flags & S_INIT_TILE) v += (double)t.init[(size_t)r * pc + c];
      if (gfull && t.gmap[r] >= 0) v += gs * gfull[(size_t)t.gmap[r] * pc + c];
      out[(size_t)r * pc + c] = v;
    }
  // all reads done before the writes (a task may overwrite its own input tile)
  for (int r = 0; r < 64; ++r)
    for (int c = 0; c < pc; ++c) {
      const T v = (T)out[(size_t)r * pc + c];
      t.C[(size_t)r * pc + c] = v;
      if (sfull && t.smap[r] >= 0) {
        double* o = sfull + (size_t)t.smap[r] * pc + c;
        *o = mv.scatter_add ? *o + (double)v : (double)v;
      }
    }
}

// Run a schedule: the groups interleaved at random step by step, the tasks of a
// step in random order.
template <typename Task, typename Run>
void run(const std::vector<std::vector<SchedStep>>& steps, const std::vector<Task>& tasks, unsigned seed, Run fn) {
  std::mt19937 rng(seed);
  std::vector<size_t> next(steps.size(), 0);
  std::vector<int> live;
  for (size_t g = 0; g < steps.size(); ++g)
    if (!steps[g].empty()) live.push_back((int)g);
  while (!live.empty()) {
    const size_t pick = rng() % live.size();
    const int g = live[pick];
    const SchedStep& st = steps[g][next[g]++];
    std::vector<int> order(st.count);
    for (int i = 0; i < st.count; ++i) order[i] = st.first + i;
    std::shuffle(order.begin(), order.end(), rng);
    for (int i : order) fn(tasks[i]);
    if (next[g] == steps[g].size()) live.erase(live.begin() + pick);
  }
}

HostCheck* H(void* p) { return static_cast<HostCheck*>(p); }

// schedule selectors
enum { SC_FACTOR = 0, SC_SOLVE_K, SC_SOLVE_A, SC_SOLVE_K8, SC_SOLVE_A8, SC_COARSE_FACTOR, SC_COARSE_SOLVE };

template <typename T>
SolveScheduleT<T>* solve_sched(WaveSched& w, int which);
template <>
SolveScheduleT<double>* solve_sched<double>(WaveSched& w, int which) {
  switch (which) {
    case SC_SOLVE_K: return &w.solveK;
    case SC_SOLVE_A: return &w.solveA;
    case SC_SOLVE_K8: return &w.solveK8;
    default: return &w.solveA8;
  }
}
template <>
SolveScheduleT<float>* solve_sched<float>(WaveSched& w, int which) {
  switch (which) {
    case SC_SOLVE_K: return &w.solveKf;
    case SC_SOLVE_A: return &w.solveAf;
    case SC_SOLVE_K8: return &w.solveK8f;
    default: return &w.solveA8f;
  }
}

int width_of(int which) { return (which == SC_SOLVE_K8 || which == SC_SOLVE_A8) ? KB : PST; }

template <typename T>
long long race_solve(HostCheck* c, int which, const MvArgs& mv, std::string* first) {
  SolveScheduleT<T>* s = solve_sched<T>(*c->w, which);
  const int pc = width_of(which);
  return race_check(s->steps, s->tasks,
                    [&](const SolveTaskT<T>& t, std::vector<Iv>& iv, int id, int g) { footprint(t, pc, mv, iv, id, g); },
                    first);
}

template <typename T>
void run_solve(HostCheck* c, int which, const MvArgs& mv, unsigned seed) {
  SolveScheduleT<T>* s = solve_sched<T>(*c->w, which);
  const int pc = width_of(which);
  run(s->steps, s->tasks, seed, [&](const SolveTaskT<T>& t) { exec(t, pc, mv); });
}

// Preconditions of the tile kernels' vector loads: every operand pointer and
// leading dimension 16-byte aligned, every inner dimension a multiple of the
// 16-byte vector width, and the schedule's summary flags true to its tasks
// (k32: every GEMM K % 32 == 0; k64: every solve K % 64 == 0; kmax).
template <typename T>
long long align_check(const ScheduleT<T>& s, std::string* first) {
  long long n = 0;
  bool k32 = true;
  auto bad = [&](const char* what, size_t i) {
    if (first->empty()) *first = std::string(what) + " of tile task " + std::to_string(i);
    ++n;
  };
  for (size_t i = 0; i < s.gemm.size(); ++i) {
    const TileTaskT<T>& t = s.gemm[i];
    for (const void* q : {(const void*)t.A, (const void*)t.B, (const void*)t.C, (const void*)t.P})
      if (q != nullptr && reinterpret_cast<uintptr_t>(q) % 16) bad("misaligned operand", i);
    for (int ld : {t.lda, t.ldb, t.ldc})
      if ((size_t)ld * sizeof(T) % 16) bad("leading dimension", i);
    if (!(t.flags & G_POTRF)) {
      if ((size_t)t.K * sizeof(T) % 16 || t.K <= 0) bad("inner dimension", i);
      if (t.K % 32) k32 = false;
    }
  }
  if (s.k32 && !k32) bad("k32 flag", 0);
  return n;
}

template <typename T>
long long align_check(const SolveScheduleT<T>& s, std::string* first) {
  long long n = 0;
  bool k64 = true;
  int kmax = 0;
  auto bad = [&](const char* what, size_t i) {
    if (first->empty()) *first = std::string(what) + " of solve task " + std::to_string(i);
    ++n;
  };
  for (size_t i = 0; i < s.tasks.size(); ++i) {
    const SolveTaskT<T>& t = s.tasks[i];
    for (const void* q : {(const void*)t.A, (const void*)t.B, (const void*)t.C, (const void*)t.init})
      if (q != nullptr && reinterpret_cast<uintptr_t>(q) % 16) bad("misaligned operand", i);
    if (t.K > 0 && ((size_t)t.lda * sizeof(T) % 16 || (size_t)t.K * sizeof(T) % 16)) bad("inner dimension", i);
    if (t.K % 64) k64 = false;
    kmax = std::max(kmax, t.K);
  }
  if (s.k64 && !k64) bad("k64 flag", 0);
  if (s.kmax != kmax) bad("kmax", 0);
  return n;
}

}  // namespace

extern "C" {

// A handle of the set-up code for a structured hexahedral mesh: a box of
// bricks (xyz NULL) or node coordinates [(NX+1)(NY+1)(NZ+1)][3]; a regular
// sx x sy partition or nboxes element boxes (x0, x1, y0, y1); nodal loads
// [(NX+1)(NY+1)(NZ+1)][3] or NULL (the end-face traction).
void* hc_create(int nx, int ny, int nz, double hx, double hy, double hz, double traction, int sx, int sy, int o,
                int os, int nboxes, const int* boxes, const double* xyz, int instances, int mixed,
                const double* load) {
  HostCheck* c = new HostCheck();
  msgfem* h = &c->h;
  h->NX = nx; h->NY = ny; h->NZ = nz;
  h->hx = hx; h->hy = hy; h->hz = hz; h->traction = traction;
  h->sx = sx; h->sy = sy; h->o = o; h->os = os;
  if (nboxes > 0) {
    h->boxes.assign(boxes, boxes + 4 * (size_t)nboxes);
    h->sx = nboxes;
    h->sy = 1;
  }
  if (xyz != nullptr) h->h_xyz.assign(xyz, xyz + 3 * (size_t)(nx + 1) * (ny + 1) * (nz + 1));
  if (load != nullptr) h->h_load.assign(load, load + 3 * (size_t)(nx + 1) * (ny + 1) * (nz + 1));
  h->S = instances > 1 ? instances : 1;
  h->mixed = mixed;
  c->st = build_problem(h);
  return c;
}

int hc_status(void* p) { return (int)H(p)->st; }
const char* hc_error(void* p) { return H(p)->h.err.c_str(); }
void hc_destroy(void* p) { delete H(p); }
int hc_num_subdomains(void* p) { return H(p)->h.N; }

// I0 I1 J0 J1 oI0 oI1 oJ0 oJ1 nxn nyn nzn npl nnode nfull nK nA bK bA floating
// loaded pin[6] n1 n2 n3 inst (29 ints)
int hc_sub_ints(void* p, int j, int* out) {
  const msgfem& h = H(p)->h;
  if (j < 0 || j >= h.N) return -1;
  const SubDev& s = h.sub[j];
  const int v[29] = {s.I0, s.I1, s.J0, s.J1, s.oI0, s.oI1, s.oJ0, s.oJ1, s.nxn, s.nyn,
                     s.nzn, s.npl, s.nnode, s.nfull, s.nK, s.nA, s.bK, s.bA, s.floating, s.loaded,
                     s.pin[0], s.pin[1], s.pin[2], s.pin[3], s.pin[4], s.pin[5], h.n1[j], h.n2[j], h.n3[j]};
  memcpy(out, v, sizeof v);
  return 0;
}

int hc_sub_arrays(void* p, int j, signed char* cls, double* mu, double* load, int* mapK, int* mapA) {
  const msgfem& h = H(p)->h;
  if (j < 0 || j >= h.N) return -1;
  const HostSub& hs = h.hsub[j];
  memcpy(cls, hs.cls.data(), hs.cls.size());
  memcpy(mu, hs.mu.data(), hs.mu.size() * sizeof(double));
  memcpy(load, hs.bload.data(), hs.bload.size() * sizeof(double));
  memcpy(mapK, hs.mapK.data(), hs.mapK.size() * sizeof(int));
  memcpy(mapA, hs.mapA.data(), hs.mapA.size() * sizeof(int));
  return 0;
}

long long hc_sub_bytes(void* p, int j) { return (long long)sub_block_bytes(&H(p)->h, j); }

// Wave grouping for a byte budget; returns the number of waves or -status.
int hc_plan_waves(void* p, double budget_bytes) {
  msgfem_status st = plan_waves(&H(p)->h, (size_t)budget_bytes);
  return st == MSGFEM_OK ? (int)H(p)->h.waves.size() : -(int)st;
}
long long hc_pool_bytes(void* p) { return (long long)H(p)->h.pool_bytes; }
int hc_wave_members(void* p, int w, int* out) {
  const msgfem& h = H(p)->h;
  if (w < 0 || w >= (int)h.waves.size()) return -1;
  for (size_t i = 0; i < h.waves[w].members.size(); ++i) out[i] = h.waves[w].members[i];
  return (int)h.waves[w].members.size();
}

// Place the members of wave w in a host pool (the product's placement) and
// build their factorisation and solve schedules.
int hc_build_wave(void* p, int w, int groups_factor, int groups_solve, int left) {
  HostCheck* c = H(p);
  msgfem* h = &c->h;
  if (w < 0 || w >= (int)h->waves.size()) return -1;
  if (c->pool == nullptr) {
    c->pool_mem.assign(h->pool_bytes + 512, 0);
    c->pool = reinterpret_cast<char*>(((uintptr_t)c->pool_mem.data() + 255) / 256 * 256);
  }
  size_t off = 0;
  for (int j : h->waves[w].members) {
    off += place_sub_blocks(h, j, c->pool + off);
    // the layer maps the solve tasks read (device copies in the library)
    h->sub[j].mapK = h->hsub[j].mapK.data();
    h->sub[j].mapA = h->hsub[j].mapA.data();
  }
  h->ngroup_factor = groups_factor;
  h->ngroup = groups_solve;
  h->factor_left = left;
  c->wave = w;
  c->w = &h->waves[w];
  build_wave_factor_schedule(h, *c->w);
  build_wave_solve_schedules(h, *c->w);
  return 0;
}

// Schedules of wave w built on a pool that is never touched (base address only):
// for counting tasks and work of full-size workloads without their memory.
int hc_build_wave_virtual(void* p, int w, int groups_factor, int groups_solve, int left) {
  HostCheck* c = H(p);
  msgfem* h = &c->h;
  if (w < 0 || w >= (int)h->waves.size()) return -1;
  char* base = reinterpret_cast<char*>((uintptr_t)1 << 40);
  size_t off = 0;
  for (int j : h->waves[w].members) {
    off += place_sub_blocks(h, j, base + off);
    h->sub[j].mapK = h->hsub[j].mapK.data();
    h->sub[j].mapA = h->hsub[j].mapA.data();
  }
  h->ngroup_factor = groups_factor;
  h->ngroup = groups_solve;
  h->factor_left = left;
  c->wave = w;
  c->w = &h->waves[w];
  c->pool = nullptr;
  build_wave_factor_schedule(h, *c->w);
  build_wave_solve_schedules(h, *c->w);
  return 0;
}

// Flops the factorisation schedule of the built wave executes: 2 * 64 * 64 * K per
// GEMM task (twice that with the 64 x 64 post-multiplication), and for a tile
// POTRF its Cholesky (64^3 / 3 multiply-adds) and inverse (64^3 / 6 multiply-adds).
double hc_factor_task_flops(void* p) {
  HostCheck* c = H(p);
  if (c->w == nullptr) return -1.0;
  double f = 0.0;
  const bool fp64 = !c->h.mixed;
  auto add = [&](int flags, int K) {
    if (flags & G_POTRF) f += 2.0 * (64.0 * 64.0 * 64.0 / 3.0 + 64.0 * 64.0 * 64.0 / 6.0);
    else
      f += 2.0 * 64.0 * 64.0 * K * ((fp64 && (flags & (G_TRIB | G_SYMC))) ? 10.0 / 16.0 : 1.0) +
           ((flags & G_POSTMUL) ? 2.0 * 64.0 * 64.0 * 64.0 * (fp64 ? 10.0 / 16.0 : 1.0) : 0.0);
  };
  if (c->h.mixed) for (const auto& t : c->w->factf.gemm) add(t.flags, t.K);
  else for (const auto& t : c->w->fact.gemm) add(t.flags, t.K);
  return f;
}

// Pointer to part `which` of subdomain j's storage: 0 D_K (then E_K), 1 Linv_K,
// 2 D_A (then E_A), 3 Linv_A.
void* hc_sub_ptr(void* p, int j, int which) {
  const msgfem& h = H(p)->h;
  const SubDev& s = h.sub[j];
  if (h.mixed) {
    const float* v[4] = {s.DKf, s.LKf, s.DAf, s.LAf};
    return (void*)v[which];
  }
  const double* v[4] = {s.DK, s.LK, s.DA, s.LA};
  return (void*)v[which];
}

// Coarse schedules over caller-owned blocks (NcPad x NcPad A^H, its inverse
// tiles, and NcPad x PST vectors b, r, y, c).
int hc_build_coarse(void* p, int ncpad, double* AH, double* AHinv, double* bH, double* rH, double* yH, double* cH) {
  HostCheck* c = H(p);
  msgfem* h = &c->h;
  if (ncpad <= 0 || ncpad % TILE) return -1;
  h->NcPad = ncpad;
  h->d_AH = AH; h->d_AHinv = AHinv; h->d_bH = bH; h->d_rH = rH; h->d_yH = yH; h->d_cH = cH;
  // the split inverse rows, as the library allocates them
  size_t tiles = 0;
  int maxc = 1;
  coarse_inverse_split_sizes(ncpad / TILE, COARSE_INV_SPLIT, &tiles, &maxc);
  c->cscr.assign(std::max<size_t>(tiles, 1) * TILE * TILE, 0.0);
  c->cid.assign((size_t)TILE * maxc * TILE, 0.0);
  for (int r = 0; r < TILE; ++r)
    for (int q = 0; q < maxc; ++q) c->cid[(size_t)r * maxc * TILE + (size_t)q * TILE + r] = 1.0;
  h->d_cscr = c->cscr.data();
  h->d_cid = c->cid.data();
  build_coarse_schedules(h);
  c->coarse = 1;
  return 0;
}

// groups, steps and tasks of a schedule
int hc_sched_shape(void* p, int which, int* out3) {
  HostCheck* c = H(p);
  const std::vector<std::vector<SchedStep>>* steps = nullptr;
  size_t ntask = 0;
  if (which == SC_COARSE_FACTOR) { steps = &c->h.cfact.steps; ntask = c->h.cfact.gemm.size(); }
  else if (which == SC_COARSE_SOLVE) { steps = &c->h.csolve.steps; ntask = c->h.csolve.tasks.size(); }
  else if (c->w == nullptr) return -1;
  else if (which == SC_FACTOR) {
    if (c->h.mixed) { steps = &c->w->factf.steps; ntask = c->w->factf.gemm.size(); }
    else { steps = &c->w->fact.steps; ntask = c->w->fact.gemm.size(); }
  } else if (c->h.mixed) {
    auto* s = solve_sched<float>(*c->w, which); steps = &s->steps; ntask = s->tasks.size();
  } else {
    auto* s = solve_sched<double>(*c->w, which); steps = &s->steps; ntask = s->tasks.size();
  }
  int nst = 0;
  for (const auto& g : *steps) nst += (int)g.size();
  out3[0] = (int)steps->size(); out3[1] = nst; out3[2] = (int)ntask;
  return 0;
}

// Race check of a schedule; src / dst: full-layout multivectors per subdomain
// (solves).  Returns the number of conflicting task pairs; msg gets the first.
long long hc_race_check(void* p, int which, double* const* src, double* const* dst, int scatter_add, char* msg,
                        int len) {
  HostCheck* c = H(p);
  std::string first;
  long long n = -1;
  MvArgs mv;
  mv.src = src; mv.dst = dst; mv.scatter_add = scatter_add;
  auto fpg = [](const auto& t, std::vector<Iv>& iv, int id, int g) { footprint(t, iv, id, g); };
  if (which == SC_COARSE_FACTOR) {
    n = race_check(c->h.cfact.steps, c->h.cfact.gemm, fpg, &first);
  } else if (which == SC_COARSE_SOLVE) {
    n = race_check(c->h.csolve.steps, c->h.csolve.tasks,
                   [&](const SolveTask& t, std::vector<Iv>& iv, int id, int g) { footprint(t, PST, mv, iv, id, g); },
                   &first);
  } else if (c->w != nullptr) {
    if (which == SC_FACTOR)
      n = c->h.mixed ? race_check(c->w->factf.steps, c->w->factf.gemm, fpg, &first)
                     : race_check(c->w->fact.steps, c->w->fact.gemm, fpg, &first);
    else
      n = c->h.mixed ? race_solve<float>(c, which, mv, &first) : race_solve<double>(c, which, mv, &first);
  }
  if (msg && len > 0) snprintf(msg, len, "%s", first.c_str());
  return n;
}

// Execute the factorisation schedule of the built wave (or the coarse one);
// returns the number of tiles found not positive definite.
int hc_run_factor(void* p, int coarse, unsigned seed) {
  HostCheck* c = H(p);
  int bad = 0;
  if (coarse) {
    run(c->h.cfact.steps, c->h.cfact.gemm, seed, [&](const GemmTask& t) { exec(t, &bad); });
  } else if (c->h.mixed) {
    run(c->w->factf.steps, c->w->factf.gemm, seed, [&](const TileTaskT<float>& t) { exec(t, &bad); });
  } else {
    run(c->w->fact.steps, c->w->fact.gemm, seed, [&](const GemmTask& t) { exec(t, &bad); });
  }
  return bad;
}

// The persistent FP32 factorisation (on: the next hc_build_wave builds its
// ticket order, one dependency group per chain).
int hc_set_persistent(void* p, int on) {
  H(p)->h.factor_persistent = on;
  return 0;
}

long long hc_persistent_tasks(void* p) {
  HostCheck* c = H(p);
  return c->w ? (long long)c->w->pmeta.size() : -1;
}

// Execute the built wave's persistent task order as `window` resident CTAs
// would: tickets are taken in order, each held ticket runs once the previous
// step of its chain has completed (the kernel's counter condition), a random
// ready one at a time.  Returns the number of tiles found not positive
// definite, -2 when no held ticket can run (a deadlock of the kernel), -3 when
// a task is missing or repeated.
int hc_run_factor_persistent(void* p, int window, unsigned seed) {
  HostCheck* c = H(p);
  if (c->w == nullptr || !c->h.mixed || c->w->pmeta.empty()) return -1;
  const std::vector<int4>& meta = c->w->pmeta;
  if (meta.size() != c->w->factf.gemm.size()) return -3;
  std::vector<char> seen(meta.size(), 0);
  for (const int4& m : meta) {
    if (m.w < 0 || (size_t)m.w >= seen.size() || seen[m.w]) return -3;
    seen[m.w] = 1;
  }
  std::vector<int> cnt(c->w->pcount, 0);
  std::mt19937 rng(seed);
  size_t next = 0;
  std::vector<size_t> held;
  int bad = 0;
  while (next < meta.size() || !held.empty()) {
    while ((int)held.size() < window && next < meta.size()) held.push_back(next++);
    std::vector<size_t> ready;
    for (size_t k = 0; k < held.size(); ++k) {
      const int4& m = meta[held[k]];
      if (m.y < 0 || cnt[m.y] >= m.z) ready.push_back(k);
    }
    if (ready.empty()) return -2;
    const size_t k = ready[rng() % ready.size()];
    const int4 m = meta[held[k]];
    exec(c->w->factf.gemm[m.w], &bad);
    ++cnt[m.x];
    held.erase(held.begin() + (long)k);
  }
  return bad;
}

int hc_run_solve(void* p, int which, double* const* src, double* const* dst, int gather_neg, int scatter_add,
                 unsigned seed) {
  HostCheck* c = H(p);
  MvArgs mv;
  mv.src = src; mv.dst = dst; mv.gather_neg = gather_neg; mv.scatter_add = scatter_add;
  if (which == SC_COARSE_SOLVE) {
    run(c->h.csolve.steps, c->h.csolve.tasks, seed, [&](const SolveTask& t) { exec(t, PST, mv); });
    return 0;
  }
  if (c->w == nullptr) return -1;
  if (c->h.mixed)
    run_solve<float>(c, which, mv, seed);
  else
    run_solve<double>(c, which, mv, seed);
  return 0;
}

// Element types of an angle field ([instances][NX NY NZ]) with optional ply
// frames ([NX NY NZ][9]); types, etype and trep sized for one type per element.
// Returns the number of types; *layered as the library decides it.
int hc_element_types(void* p, const double* angles, const double* frames, int* layered, double* types, int* etype,
                     int* trep) {
  msgfem* h = &H(p)->h;
  const size_t nel = (size_t)h->NX * h->NY * h->NZ, ntot = nel * h->S;
  h->h_angles.assign(angles, angles + ntot);
  if (frames != nullptr) h->h_frame.assign(frames, frames + 9 * nel);
  else h->h_frame.clear();
  bool lay = false;
  std::vector<double> ty;
  std::vector<int> et, tr;
  element_types(h, lay, ty, et, tr);
  *layered = lay ? 1 : 0;
  memcpy(types, ty.data(), ty.size() * sizeof(double));
  memcpy(etype, et.data(), et.size() * sizeof(int));
  memcpy(trep, tr.data(), tr.size() * sizeof(int));
  return (int)ty.size();
}

// Coarse pairs (s, t, x0, x1, y0, y1): the node box of Omega_s cap Omega*_t over
// which the block A^H_{st} is accumulated.  out: 6 ints per pair (NULL: count only).
int hc_pairs(void* p, int* out) {
  const msgfem& h = H(p)->h;
  if (out != nullptr)
    for (size_t i = 0; i < h.pairs.size(); ++i) {
      const CoarsePair& c = h.pairs[i];
      const int v[6] = {c.s, c.t, c.x0, c.x1, c.y0, c.y1};
      memcpy(out + 6 * i, v, sizeof v);
    }
  return (int)h.pairs.size();
}

long long hc_align_check(void* p, int which, char* msg, int len) {
  HostCheck* c = H(p);
  std::string first;
  long long n = -1;
  if (which == SC_COARSE_FACTOR) n = align_check(c->h.cfact, &first);
  else if (which == SC_COARSE_SOLVE) n = align_check(c->h.csolve, &first);
  else if (c->w == nullptr) n = -1;
  else if (which == SC_FACTOR) n = c->h.mixed ? align_check(c->w->factf, &first) : align_check(c->w->fact, &first);
  else n = c->h.mixed ? align_check(*solve_sched<float>(*c->w, which), &first)
                      : align_check(*solve_sched<double>(*c->w, which), &first);
  if (msg && len > 0) snprintf(msg, len, "%s", first.c_str());
  return n;
}

// Preconditions of the TMA-filled solve ring (k_solve_tma) on the FP32
// 8-column solve schedules, the conditions the kernel checks on the device
// before its first copy: a task with an inner dimension reads one 64-row slab
// of one of its subdomain's four FP32 arrays (D|E and inverse of K, then of
// A11), with that array's row stride, a column that is a multiple of 4 floats
// (16 bytes) and every stage inside the array.  Returns the violations.
long long hc_tma_check(void* p, int which, char* msg, int len) {
  HostCheck* c = H(p);
  if (c->w == nullptr || !c->h.mixed) return -1;
  const SolveScheduleT<float>* s = solve_sched<float>(*c->w, which);
  long long n = 0;
  std::string first;
  for (size_t i = 0; i < s->tasks.size(); ++i) {
    const SolveTaskT<float>& t = s->tasks[i];
    if (t.K <= 0) continue;
    bool ok = false;
    if (t.sub >= 0 && t.sub < c->h.N) {
      const SubDev& sd = c->h.sub[t.sub];
      const float* base[4] = {sd.DKf, sd.LKf, sd.DAf, sd.LAf};
      const int b[4] = {sd.bK, sd.bK, sd.bA, sd.bA};
      const int rows[4] = {(2 * sd.nzn - 1) * sd.bK, sd.nzn * sd.bK, (2 * sd.nzn - 1) * sd.bA, sd.nzn * sd.bA};
      for (int m = 0; m < 4 && !ok; ++m) {
        if (base[m] == nullptr || t.A < base[m]) continue;
        const long long off = t.A - base[m];
        if (off >= (long long)rows[m] * b[m]) continue;
        const int y = (int)(off / b[m]), x = (int)(off % b[m]);
        const bool tr = (t.flags & S_TRANSA) != 0;
        const int w = tr ? 64 : t.K, hgt = tr ? t.K : 64;
        ok = t.lda == b[m] && x % 4 == 0 && x + w <= b[m] && y + hgt <= rows[m] && t.K % 64 == 0;
      }
    }
    if (!ok) {
      if (first.empty()) first = "solve task " + std::to_string(i) + " outside the TMA preconditions";
      ++n;
    }
  }
  if (msg && len > 0) snprintf(msg, len, "%s", first.c_str());
  return n;
}

// A planted scheduling mistake, for checking the race check itself: step s of
// group g merged with step s + 1 (two dependent launches made one).
int hc_merge_steps(void* p, int which, int g, int s) {
  HostCheck* c = H(p);
  std::vector<std::vector<SchedStep>>* steps = nullptr;
  if (which == SC_FACTOR && c->w) steps = c->h.mixed ? &c->w->factf.steps : &c->w->fact.steps;
  else if (c->w && which >= SC_SOLVE_K && which <= SC_SOLVE_A8)
    steps = c->h.mixed ? &solve_sched<float>(*c->w, which)->steps : &solve_sched<double>(*c->w, which)->steps;
  if (steps == nullptr || g < 0 || g >= (int)steps->size() || s < 0 || s + 1 >= (int)(*steps)[g].size()) return -1;
  auto& v = (*steps)[g];
  if (v[s].first + v[s].count != v[s + 1].first) return -1;
  v[s].count += v[s + 1].count;
  v.erase(v.begin() + s + 1);
  return 0;
}

}  // extern "C"
