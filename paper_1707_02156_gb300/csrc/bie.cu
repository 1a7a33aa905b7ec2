// C ABI entry points: context and plan caches, transforms, geometry set-up, the layer-operator
// applies (Eq. main_eq) and the GMRES solve (Sec. 6).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <initializer_list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "dfloat.cuh"
#include "interdrop.h"
#include "near.h"
#include "offsurface.h"
#include "internal.cuh"
#include "tables.h"

namespace bie {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

static const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------------------------
template <typename T>
struct DevBuf {
  T* ptr = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    n = 0;
  }
  int alloc(size_t count) {
    if (count <= n && ptr) return BIE_OK;
    release();
    if (count == 0) return BIE_OK;
    cudaError_t e = cudaMalloc(&ptr, count * sizeof(T));
    if (e != cudaSuccess) {
      ptr = nullptr;
      set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
      return BIE_ENOMEM;
    }
    n = count;
    return BIE_OK;
  }
  int upload(const T* host, size_t count) {
    BIE_TRY(alloc(count));
    if (count) BIE_CUDA_TRY(cudaMemcpy(ptr, host, count * sizeof(T), cudaMemcpyHostToDevice));
    return BIE_OK;
  }
  int upload(const std::vector<T>& v) { return upload(v.data(), v.size()); }
};

template <typename T>
static int upload_as(DevBuf<T>& dst, const std::vector<double>& v) {
  std::vector<T> tmp(v.begin(), v.end());
  return dst.upload(tmp);
}

// ---------------------------------------------------------------------------------------------
// plans: tables for coefficients of degree p on the grid of degree P
// ---------------------------------------------------------------------------------------------
struct Plan {
  int p = 0, P = 0;
  DevBuf<double> T0, T1, T2, A, cs, wsin, wsq;
  DevBuf<float> T0f, csf;
  DevBuf<dff> csdf;
  template <typename R>
  const R* T0_() const;
  template <typename R>
  const R* cs_() const;
};
template <>
const double* Plan::T0_<double>() const {
  return T0.ptr;
}
template <>
const float* Plan::T0_<float>() const {
  return T0f.ptr;
}
template <>
const double* Plan::cs_<double>() const {
  return cs.ptr;
}
template <>
const float* Plan::cs_<float>() const {
  return csf.ptr;
}
template <>
const dff* Plan::cs_<dff>() const {
  return csdf.ptr;
}

struct WigPlan {  // rotation blocks for the p+1 latitudes of the degree-p grid
  int p = 0;
  long long stride = 0;
  DevBuf<double> blk;
  DevBuf<float> blkf;
  DevBuf<dff> blkdf;
  template <typename R>
  const R* blk_() const;
};
template <>
const double* WigPlan::blk_<double>() const {
  return blk.ptr;
}
template <>
const float* WigPlan::blk_<float>() const {
  return blkf.ptr;
}
template <>
const dff* WigPlan::blk_<dff>() const {
  return blkdf.ptr;
}

}  // namespace bie

struct bie_ctx {
  bie_config cfg;
  int sms = 0;  // streaming multiprocessors of the device (sizes the work lists)
  struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<std::pair<std::string, size_t>> recs;  // name, index of the start event
  } prof;
  std::mutex mu;
  std::map<std::pair<int, int>, std::unique_ptr<bie::Plan>> plans;
  std::map<int, std::unique_ptr<bie::WigPlan>> wigs;
  bie::DevBuf<double> scratch;  // analysis workspace
  // pair-kernel variant chosen at earlier geometries: degrees, self-grid degrees, U, pair count, variant
  struct Tuned {
    std::vector<int> p, pq;
    int up;
    long long pairs;
    int tpt;
  };
  std::vector<Tuned> tuned;
};

namespace bie {

static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches += n; }

// Per-phase CUDA-event timing on the launching stream (enabled by bie_profile).
struct Phase {
  bie_ctx* ctx;
  cudaStream_t s;
  size_t idx = (size_t)-1;
  Phase(bie_ctx* c, const char* name, cudaStream_t st) : ctx(c), s(st) {
    if (!ctx || !ctx->prof.on) return;
    auto& P = ctx->prof;
    while (P.pool.size() < P.used + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      P.pool.push_back(e);
    }
    idx = P.used;
    P.used += 2;
    P.recs.emplace_back(name, idx);
    cudaEventRecord(P.pool[idx], s);
  }
  ~Phase() {
    if (idx != (size_t)-1) cudaEventRecord(ctx->prof.pool[idx + 1], s);
  }
};

int ctx_device(const bie_ctx* ctx) { return ctx->cfg.device; }

static int get_plan(bie_ctx* ctx, int p, int P, Plan** out) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto key = std::make_pair(p, P);
  auto it = ctx->plans.find(key);
  if (it != ctx->plans.end()) {
    *out = it->second.get();
    return BIE_OK;
  }
  std::unique_ptr<Plan> pl(new Plan());
  pl->p = p;
  pl->P = P;
  std::vector<double> v;
  legendre_table(p, P, 0, v);
  BIE_TRY(pl->T0.upload(v));
  BIE_TRY(upload_as(pl->T0f, v));
  legendre_table(p, P, 1, v);
  BIE_TRY(pl->T1.upload(v));
  legendre_table(p, P, 2, v);
  BIE_TRY(pl->T2.upload(v));
  analysis_table(p, P, v);
  BIE_TRY(pl->A.upload(v));
  phase_table(p, P, v);
  BIE_TRY(pl->cs.upload(v));
  BIE_TRY(upload_as(pl->csf, v));
  BIE_TRY(upload_as(pl->csdf, v));
  std::vector<double> t, w, ws;
  gauss_legendre(P + 1, t, w);
  singular_weights(P, ws);
  std::vector<double> wsin(P + 1), wsq(P + 1);
  for (int j = 0; j <= P; ++j) {
    double s = std::sqrt((1.0 - t[j]) * (1.0 + t[j]));
    wsin[j] = kPi / (P + 1) * w[j] / s;
    wsq[j] = ws[j] / s;
  }
  BIE_TRY(pl->wsin.upload(wsin));
  BIE_TRY(pl->wsq.upload(wsq));
  *out = pl.get();
  ctx->plans[key] = std::move(pl);
  return BIE_OK;
}

static int get_wig(bie_ctx* ctx, int p, WigPlan** out) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->wigs.find(p);
  if (it != ctx->wigs.end()) {
    *out = it->second.get();
    return BIE_OK;
  }
  std::unique_ptr<WigPlan> wp(new WigPlan());
  wp->p = p;
  wp->stride = wigner_block_stride(p);
  std::vector<double> t, w;
  gauss_legendre(p + 1, t, w);
  std::vector<double> blk((size_t)(p + 1) * wp->stride);
  for (int a = 0; a <= p; ++a) wigner_blocks(p, std::acos(t[a]), blk.data() + (size_t)a * wp->stride);
  BIE_TRY(wp->blk.upload(blk));
  BIE_TRY(upload_as(wp->blkf, blk));
  BIE_TRY(upload_as(wp->blkdf, blk));
  *out = wp.get();
  ctx->wigs[p] = std::move(wp);
  return BIE_OK;
}

static inline long long ncoef(int p) { return (long long)(p + 1) * (p + 1); }
static inline long long ngrid(int P) { return (long long)(P + 1) * (2 * P + 2); }

static int check_degrees(int ndrop, const int* p) {
  if (ndrop <= 0 || !p) {
    set_error("ndrop must be positive and p non-null");
    return BIE_EINVAL;
  }
  for (int d = 0; d < ndrop; ++d)
    if (p[d] < 1 || p[d] > BIE_MAX_P) {
      set_error("degree out of range [1, BIE_MAX_P]");
      return BIE_EINVAL;
    }
  return BIE_OK;
}

}  // namespace bie

// ---------------------------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------------------------
namespace bie {
struct Krylov;
}

struct bie_geom {
  bie_ctx* ctx = nullptr;
  int ndrop = 0;
  std::vector<int> p, pq;
  std::vector<double> lambda;
  std::vector<long long> coef_off;  // start of drop d's [3][(p+1)^2] block (doubles)
  std::vector<long long> tgt_off;   // first target of drop d
  long long ncoef_total = 0, ntarget = 0;
  bie::DevBuf<double> xcoef;        // copy of the shape coefficients
  bie::DevBuf<double> rec_std;      // [drop][7][N_g] targets / standard-grid sources
  bie::DevBuf<double> vals;         // [drop][3][N_g] apply values at the grid targets
  bie::DevBuf<double> lamc;         // lambda of the drop owning each coefficient
  struct Group {
    int p = 0, pq = 0;
    std::vector<int> drops;
    bie::DevBuf<long long> foff3, goff3, val_off, roff;  // roff: 7 * first target, per group drop
    bie::DevBuf<double> wS, wD, wSraw, wDraw;
    bie::DevBuf<double> cache64;            // [gdrop][N_g][7][nq] rotated geometry (Sec. 2.2)
    bie::DevBuf<float> cache32;             // FP32 copy, made on the first direct-form mixed apply
    bie::DevBuf<long long> src_off_std, src_off_up;  // first source of each drop on the two grids
    bie::DevBuf<double> qk64[2];            // projected kernel factors of every target, S and D
    bie::DevBuf<float> qk32[2];
    bie::DevBuf<bie::dff> qkdf[2];          // double-float copy, made on the first BIE_DF apply
  };
  std::vector<std::unique_ptr<Group>> groups;
  struct GraphSlot {
    bool warm = false;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
  };
  std::map<int, GraphSlot> graphs;       // captured applies by (flags, kind)
  bie::DevBuf<double> gin, gout;          // fixed input / output of the captured applies
  cudaStream_t cap_stream = nullptr;
  bie::Krylov* kry = nullptr;  // solve workspace, kept between solves
  bie_geom_info info{};
  // inter-drop data (ndrop > 1), Sec. 2.3
  std::vector<double> centre, bound, hdrop, volume;
  std::vector<long long> up_off, up_n;
  std::vector<int> up_P;
  long long nup_total = 0;
  bie::DevBuf<double> rec_up;                       // [drop][7][N_up] upsampled-grid records
  bie::DevBuf<double> sX64, sN64, uX64, uN64, sQ64, uQ64;  // sources: positions rel. centre, normals, weighted density
  bie::DevBuf<float> sX32, sN32, uX32, uN32, sQ32, uQ32;
  bie::DevBuf<double> syn64;                        // synthesis temporaries for the source densities
  bie::DevBuf<float> syn32;
  bie::DevBuf<bie::PairItem> items;
  bie::DevBuf<int> blk_item, tile_n, tile_drop, tile_blk, tdrop, ngd;
  bie::DevBuf<long long> tile_t0, tgt_loc, toff, val_off_all;
  bie::DevBuf<double> centre_d, partial, wS_all, wD_all, wSr_all, wDr_all;
  int nblk = 0, ntile = 0;
  bool interdrop_ready = false;  // inter-drop data built: at set-up when ndrop > 1, else at the first off-surface evaluation
  int tpt32 = 2, tpt64 = 2;                         // targets per thread of the pair kernel (autotuned FP32)
  bie::DevBuf<float> eo32;                          // tensor-core self path: rotated sums
  bie::DevBuf<unsigned> g32;                        // and the split phase-shifted coefficients
  std::vector<std::pair<long long, int>> near;      // (target, source drop) pairs in Omega_2
  // near-singular step (Omega_2), Sec. 2.3
  int nnear_tgt = 0;
  bie::DevBuf<bie::NearPair> npairs;
  bie::DevBuf<int> ntbeg, ngrid_l, pdeg_d;
  bie::DevBuf<double> npts, ncv, selfvals, selfcoef, hdrop_d;
  bie::DevBuf<long long> coef_off_d, up_off_d, up_n_d;
};

namespace bie {

static const long long kWorkBudget = 3LL << 30;  // bytes of set-up temporaries per chunk

// Galerkin projection of the values of every degree group, one launch.
static int analyze_groups(bie_ctx* ctx, bie_geom* g, const double* vals, double* out, cudaStream_t s) {
  std::vector<AnaGroup> ag;
  for (auto& Gp : g->groups) {
    auto& G = *Gp;
    Plan* pl;
    BIE_TRY(get_plan(ctx, G.p, G.p, &pl));
    AnaGroup a{};
    a.nfield = (long long)G.drops.size() * 3;
    a.grid_off = G.goff3.ptr;
    a.coef_off = G.foff3.ptr;
    a.cs = pl->cs.ptr;
    a.A = pl->A.ptr;
    a.p = G.p;
    ag.push_back(a);
  }
  std::sort(ag.begin(), ag.end(), [](const AnaGroup& x, const AnaGroup& y) { return x.p > y.p; });
  Phase ph(ctx, "analyze", s);
  return launch_analyze_fused(ag, vals, out, s);
}

// The direct form serves a group when the configuration asks for it, or when the projected form's
// per-target factors would not fit in shared memory while they are built.
static bool group_uses_direct(const bie_ctx* ctx, const bie_geom::Group& G) {
  return ctx->cfg.self_direct != 0 || kernel_proj_smem(G.p, G.pq) > 227 * 1024;
}

// Projected-form kernel factors of one group, built from the FP64 rotated-grid cache.
static int ensure_qk(bie_ctx* ctx, bie_geom::Group& G, int kind, cudaStream_t s) {
  if (G.qk64[kind].ptr) return BIE_OK;
  Plan* pl;
  BIE_TRY(get_plan(ctx, G.p, G.pq, &pl));
  const long long nt = (long long)G.drops.size() * ngrid(G.p);
  const long long n = nt * 6 * (long long)(G.p + 1) * (G.p + 2);
  BIE_TRY(G.qk64[kind].alloc(n));
  BIE_TRY(G.qk32[kind].alloc(n));
  Phase ph(ctx, "kernel_proj", s);
  return launch_kernel_proj(kind, G.cache64.ptr, nt, G.p, G.pq, pl->cs.ptr, pl->T0.ptr, G.qk64[kind].ptr,
                            G.qk32[kind].ptr, s);
}

// Projected factors of one group in the arithmetic type R (the double-float copy is split from the
// FP64 factors on first use).
template <typename R>
static int qk_of(bie_geom::Group& G, int kind, cudaStream_t s, const R** out);
template <>
int qk_of<double>(bie_geom::Group& G, int kind, cudaStream_t, const double** out) {
  *out = G.qk64[kind].ptr;
  return BIE_OK;
}
template <>
int qk_of<float>(bie_geom::Group& G, int kind, cudaStream_t, const float** out) {
  *out = G.qk32[kind].ptr;
  return BIE_OK;
}
template <>
int qk_of<dff>(bie_geom::Group& G, int kind, cudaStream_t s, const dff** out) {
  if (!G.qkdf[kind].ptr) {
    BIE_TRY(G.qkdf[kind].alloc(G.qk64[kind].n));
    BIE_TRY(launch_split_dff(G.qk64[kind].ptr, G.qkdf[kind].ptr, (long long)G.qk64[kind].n, s));
  }
  *out = G.qkdf[kind].ptr;
  return BIE_OK;
}
template <typename R>
static const char* self_phase_name() {
  return std::is_same<R, float>::value ? "self_proj_f32" : std::is_same<R, dff>::value ? "self_proj_df" : "self_proj_f64";
}

// Singular self part of every drop (Sec. 2.2): one launch for every projected-form degree group
// (direct-form groups one launch each; in double-float arithmetic those run in FP64).
template <typename R>
static int self_apply(bie_geom* g, int kind, bool raw, const double* dens, cudaStream_t s) {
  using RD = typename std::conditional<std::is_same<R, dff>::value, double, R>::type;
  bie_ctx* ctx = g->ctx;
  // the projected form keeps its per-target factors in shared memory while they are built; groups
  // whose factors do not fit there use the direct form
  auto use_direct = [&](const bie_geom::Group& G) { return group_uses_direct(ctx, G); };
  std::vector<SelfGroup<R>> proj;
  for (auto& Gp : g->groups) {
    auto& G = *Gp;
    const int p = G.p, pq = G.pq;
    const bool direct = use_direct(G);
    Plan *pl, *pp;
    WigPlan* wp;
    BIE_TRY(get_plan(ctx, p, pq, &pl));
    BIE_TRY(get_plan(ctx, p, p, &pp));
    BIE_TRY(get_wig(ctx, p, &wp));
    const double* wts = kind == 0 ? (raw ? G.wSraw.ptr : G.wS.ptr) : (raw ? G.wDraw.ptr : G.wD.ptr);
    const long long nd = (long long)G.drops.size();
    if (direct) {
      if (sizeof(RD) == 4 && !G.cache32.ptr) {
        BIE_TRY(G.cache32.alloc(G.cache64.n));
        BIE_TRY(launch_to_float(G.cache64.ptr, G.cache32.ptr, (long long)G.cache64.n, s));
      }
      const RD* cache = sizeof(RD) == 8 ? reinterpret_cast<const RD*>(G.cache64.ptr)
                                        : reinterpret_cast<const RD*>(G.cache32.ptr);
      Phase ph(ctx, sizeof(RD) == 8 ? "self_direct_f64" : "self_direct_f32", s);
      BIE_TRY(launch_self_direct<RD>(kind, dens, G.foff3.ptr, nd, p, pq, wp->blk_<RD>(), wp->stride,
                                     pp->cs_<RD>(), pl->T0_<RD>(), pl->cs_<RD>(), cache, wts, G.val_off.ptr,
                                     g->vals.ptr, sizeof(RD) == 8 ? 96 * 1024 : 40 * 1024, s));
    } else {
      BIE_TRY(ensure_qk(ctx, G, kind, s));
      SelfGroup<R> sg{};
      sg.ndrop = nd;
      sg.foff3 = G.foff3.ptr;
      sg.wblk = wp->blk_<R>();
      sg.wstride = wp->stride;
      sg.ph = pp->cs_<R>();
      BIE_TRY(qk_of<R>(G, kind, s, &sg.Q));
      sg.wts = wts;
      sg.val_off = G.val_off.ptr;
      sg.p = p;
      proj.push_back(sg);
    }
  }
  if (!proj.empty()) {  // every projected-form group in one launch; it reads the FP64 density directly
    Phase ph(ctx, self_phase_name<R>(), s);
    if constexpr (std::is_same<R, float>::value) {
      if (ctx->cfg.tensor_rotation) {
        // degrees whose rotation block fits one SM's shared memory go to the tensor cores, the rest
        // (above 58) to the CUDA-core kernel
        std::vector<SelfGroup<R>> tc, cc;
        for (const auto& sg : proj) (self_tc_fits(sg.p) ? tc : cc).push_back(sg);
        if (!tc.empty()) {
          // E/O sums of a chunk of drops kept within 32 MB, so that they stay in L2 between the kernels
          const long long budget = 8LL << 20;
          BIE_TRY(g->eo32.alloc((size_t)self_tc_eo_floats(tc, budget)));
          BIE_TRY(g->g32.alloc((size_t)self_tc_g_floats(tc, budget)));
          BIE_TRY(launch_self_tc(tc, dens, g->vals.ptr, g->eo32.ptr, g->g32.ptr, budget, s));
        }
        if (!cc.empty()) BIE_TRY((launch_self_proj<R, double>(cc, dens, g->vals.ptr, s)));
        return BIE_OK;
      }
    }
    BIE_TRY((launch_self_proj<R, double>(proj, dens, g->vals.ptr, s)));
  }
  return BIE_OK;
}

template <typename R>
static int interdrop_apply(bie_geom* g, int kind, bool raw, const double* dens, cudaStream_t s, bool df = false);
static int near_apply(bie_geom* g, int kind, bool raw, int prec, const double* dens, cudaStream_t s);
static int near_snapshot(bie_geom* g, cudaStream_t s);

static int layer_apply_eager(bie_ctx* ctx, const bie_geom* gc, int kind, const double* dens, double* out,
                             int precision, cudaStream_t s) {
  bie_geom* g = const_cast<bie_geom*>(gc);
  if (!ctx || !g || !dens || !out) {
    set_error("null argument");
    return BIE_EINVAL;
  }
  const bool raw = (precision & BIE_RAW) != 0;
  const int prec = precision & 0xff;
  if (prec != BIE_FP64 && prec != BIE_MIXED && prec != BIE_DF) {
    set_error("precision must be BIE_FP64, BIE_MIXED or BIE_DF");
    return BIE_EINVAL;
  }
  if (prec == BIE_MIXED)
    BIE_TRY(self_apply<float>(g, kind, raw, dens, s));
  else if (prec == BIE_DF)
    BIE_TRY(self_apply<dff>(g, kind, raw, dens, s));
  else
    BIE_TRY(self_apply<double>(g, kind, raw, dens, s));
  if (g->ndrop > 1) {
    if (!g->near.empty()) BIE_TRY(near_snapshot(g, s));
    if (prec == BIE_MIXED)
      BIE_TRY(interdrop_apply<float>(g, kind, raw, dens, s));
    else
      BIE_TRY(interdrop_apply<double>(g, kind, raw, dens, s, prec == BIE_DF));
    // the FP64 source densities of BIE_DF are already in place
    BIE_TRY(near_apply(g, kind, raw, prec == BIE_DF ? BIE_FP64 : prec, dens, s));
  }
  if (precision & BIE_GRID_OUT) {
    BIE_CUDA_TRY(cudaMemcpyAsync(out, g->vals.ptr, 3 * g->ntarget * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return BIE_OK;
  }
  BIE_TRY(analyze_groups(ctx, g, g->vals.ptr, out, s));
  return BIE_OK;
}

// An apply (kind, flags) that has run once eagerly is captured into a CUDA graph on an internal
// stream, reading and writing fixed internal buffers; later calls copy the input in, replay the graph
// on the caller's stream and copy the result out.  The eager run performs every lazy allocation, so
// nothing allocates or synchronises inside the capture.
static int layer_apply(bie_ctx* ctx, const bie_geom* gc, int kind, const double* dens, double* out, int precision,
                       cudaStream_t s) {
  bie_geom* g = const_cast<bie_geom*>(gc);
  if (!ctx || !g || !dens || !out) {
    set_error("null argument");
    return BIE_EINVAL;
  }
  // per-phase profiling needs the kernels launched one by one
  if (!ctx->cfg.use_graphs || ctx->prof.on) return layer_apply_eager(ctx, g, kind, dens, out, precision, s);
  const int key = (precision & 0x3ff) * 2 + kind;
  auto& slot = g->graphs[key];
  const size_t nin = g->ncoef_total;
  const size_t nout = (precision & BIE_GRID_OUT) ? 3 * g->ntarget : g->ncoef_total;
  if (!slot.exec) {
    if (!slot.warm) {  // first call with this key: eager, performs the lazy allocations
      BIE_TRY(layer_apply_eager(ctx, g, kind, dens, out, precision, s));
      slot.warm = true;
      return BIE_OK;
    }
    BIE_TRY(g->gin.alloc(std::max(g->ncoef_total, 3 * g->ntarget)));
    BIE_TRY(g->gout.alloc(std::max(g->ncoef_total, 3 * g->ntarget)));
    if (!g->cap_stream) BIE_CUDA_TRY(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    BIE_CUDA_TRY(cudaStreamSynchronize(s));
    const bool prof = ctx->prof.on;
    ctx->prof.on = false;  // no event records inside the graph
    const long long l0 = bie_launch_count();
    BIE_CUDA_TRY(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeRelaxed));
    const int st = layer_apply_eager(ctx, g, kind, g->gin.ptr, g->gout.ptr, precision, g->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(g->cap_stream, &graph);
    ctx->prof.on = prof;
    if (st != BIE_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ce != cudaSuccess) {
      set_error(std::string("graph capture: ") + cudaGetErrorString(ce));
      return BIE_ECUDA;
    }
    slot.launches = bie_launch_count() - l0;
    count_launch(-(int)slot.launches);  // captured, not run
    const cudaError_t ie = cudaGraphInstantiate(&slot.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      slot.exec = nullptr;
      set_error(std::string("graph instantiate: ") + cudaGetErrorString(ie));
      return BIE_ECUDA;
    }
  }
  Phase ph(ctx, "apply_graph", s);
  BIE_CUDA_TRY(cudaMemcpyAsync(g->gin.ptr, dens, nin * sizeof(double), cudaMemcpyDeviceToDevice, s));
  BIE_CUDA_TRY(cudaGraphLaunch(slot.exec, s));
  count_launch((int)slot.launches);
  BIE_CUDA_TRY(cudaMemcpyAsync(out, g->gout.ptr, nout * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return BIE_OK;
}

// ---------------------------------------------------------------------------------------------
// geometry set-up
// ---------------------------------------------------------------------------------------------
// x, x_theta, x_phi of ncomp=3 fields on the grid of degree P from coefficients of degree p.
static int synth_xderivs(bie_ctx* ctx, const double* coef, const long long* field_off, long long coef_stride,
                         long long nfield, int p, int P, double* H, double* X, double* Xt, double* Xp,
                         cudaStream_t s) {
  Plan* pl;
  BIE_TRY(get_plan(ctx, p, P, &pl));
  const long long N = ngrid(P);
  BIE_TRY((launch_leg_synth<double, double>(coef, field_off, coef_stride, nfield, p, pl->T0.ptr, P + 1, H, 0, s)));
  BIE_TRY((launch_phi_synth<double, double>(H, nfield, p, P, pl->cs.ptr, X, nullptr, N, s)));
  BIE_TRY((launch_leg_synth<double, double>(coef, field_off, coef_stride, nfield, p, pl->T0.ptr, P + 1, H, 1, s)));
  BIE_TRY((launch_phi_synth<double, double>(H, nfield, p, P, pl->cs.ptr, Xp, nullptr, N, s)));
  BIE_TRY((launch_leg_synth<double, double>(coef, field_off, coef_stride, nfield, p, pl->T1.ptr, P + 1, H, 0, s)));
  BIE_TRY((launch_phi_synth<double, double>(H, nfield, p, P, pl->cs.ptr, Xt, nullptr, N, s)));
  return BIE_OK;
}

static int setup_group(bie_ctx* ctx, bie_geom* g, bie_geom::Group& G, cudaStream_t s) {
  const int p = G.p, pq = G.pq;
  const long long ng = ngrid(p), nq = ngrid(pq), nc = ncoef(p);
  const int nd = (int)G.drops.size();
  // offsets
  std::vector<long long> foff3(3 * nd), goff3(3 * nd), voff(nd), roff(nd);
  std::vector<double> wS(nd), wD(nd), wSr(nd), wDr(nd);
  for (int i = 0; i < nd; ++i) {
    int d = G.drops[i];
    for (int c = 0; c < 3; ++c) {
      foff3[3 * i + c] = g->coef_off[d] + c * nc;
      goff3[3 * i + c] = 3 * g->tgt_off[d] + c * ng;
    }
    voff[i] = 3 * g->tgt_off[d];
    roff[i] = 7 * g->tgt_off[d];
    wS[i] = -1.0 / (4 * kPi);
    wD[i] = (g->lambda[d] - 1.0) / (4 * kPi);
    wSr[i] = 1.0 / (8 * kPi);
    wDr[i] = 1.0 / (4 * kPi);
  }
  BIE_TRY(G.foff3.upload(foff3));
  BIE_TRY(G.goff3.upload(goff3));
  BIE_TRY(G.val_off.upload(voff));
  BIE_TRY(G.roff.upload(roff));
  BIE_TRY(G.wS.upload(wS));
  BIE_TRY(G.wD.upload(wD));
  BIE_TRY(G.wSraw.upload(wSr));
  BIE_TRY(G.wDraw.upload(wDr));

  // standard grid: targets and regular-rule sources, one drop at a time
  {
    Phase ph(ctx, "setup_surface", s);
    Plan* pl;
    BIE_TRY(get_plan(ctx, p, p, &pl));
    DevBuf<double> tmp;
    BIE_TRY(tmp.alloc(3 * (p + 1) * (p + 1) * 2 + 9 * ng));
    double* H = tmp.ptr;
    double* X = H + 3 * (p + 1) * (p + 1) * 2;
    for (int i = 0; i < nd; ++i) {
      int d = G.drops[i];
      BIE_TRY(synth_xderivs(ctx, g->xcoef.ptr + g->coef_off[d], nullptr, nc, 3, p, p, H, X, X + 3 * ng,
                            X + 6 * ng, s));
      BIE_TRY(launch_surface(X, X + 3 * ng, X + 6 * ng, 1, p, pl->wsin.ptr, g->rec_std.ptr + 7 * g->tgt_off[d], s));
    }
    BIE_CUDA_TRY(cudaStreamSynchronize(s));
  }

  // rotated-grid cache of the singular rule (Sec. 2.2), chunked over drops
  Phase ph(ctx, "setup_rotcache", s);
  Plan *pl, *pp;
  WigPlan* wp;
  BIE_TRY(get_plan(ctx, p, pq, &pl));
  BIE_TRY(get_plan(ctx, p, p, &pp));
  BIE_TRY(get_wig(ctx, p, &wp));
  BIE_TRY(G.cache64.alloc((size_t)nd * ng * 7 * nq));
  const long long per = ng * 3 * nc + ng * 3 * (long long)(p + 1) * (pq + 1) * 2 + 3 * ng * 3 * nq;
  int chunk = (int)std::max(1LL, std::min<long long>(nd, (2 * kWorkBudget) / (8 * per)));
  DevBuf<double> work;
  BIE_TRY(work.alloc((size_t)chunk * per));
  for (int c0 = 0; c0 < nd; c0 += chunk) {
    const int cn = std::min(chunk, nd - c0);
    double* RC = work.ptr;
    double* H = RC + cn * ng * 3 * nc;
    double* X = H + cn * ng * 3 * (long long)(p + 1) * (pq + 1) * 2;
    double* Xt = X + cn * ng * 3 * nq;
    double* Xp = Xt + cn * ng * 3 * nq;
    // x coefficients of the chunk's drops: field offsets into the geometry's copy
    BIE_TRY((launch_rotate<double, double>(g->xcoef.ptr, G.foff3.ptr + 3 * c0, 3, cn, p, wp->blk.ptr, wp->stride,
                                           p + 1, 2 * p + 2, pp->cs.ptr, RC, ng * 3 * nc, s)));
    BIE_TRY(synth_xderivs(ctx, RC, nullptr, nc, cn * ng * 3, p, pq, H, X, Xt, Xp, s));
    // the targets x0 of the chunk's drops, wherever each drop's records lie (a degree group's drops
    // are in general not adjacent in rec_std)
    BIE_TRY(launch_rotgeo<double>(X, Xt, Xp, cn, (int)ng, pq, g->rec_std.ptr, G.roff.ptr + c0, pl->wsq.ptr,
                                  G.cache64.ptr + (long long)c0 * ng * 7 * nq, s));
    BIE_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return BIE_OK;
}


// ---------------------------------------------------------------------------------------------
// inter-drop set-up (Sec. 2.3): centres, volumes and mean radii, upsampled grids, source records,
// region classification, and the balanced work list of the pair sums
// ---------------------------------------------------------------------------------------------
static int drop_records(bie_ctx* ctx, bie_geom* g, int d, int P, double* rec, cudaStream_t s) {
  const int p = g->p[d];
  Plan* pl;
  BIE_TRY(get_plan(ctx, p, P, &pl));
  const long long N = ngrid(P);
  DevBuf<double> tmp;
  BIE_TRY(tmp.alloc(3 * (p + 1) * (size_t)(P + 1) * 2 + 9 * N));
  double* H = tmp.ptr;
  double* X = H + 3 * (p + 1) * (long long)(P + 1) * 2;
  BIE_TRY(synth_xderivs(ctx, g->xcoef.ptr + g->coef_off[d], nullptr, ncoef(p), 3, p, P, H, X, X + 3 * N, X + 6 * N,
                        s));
  BIE_TRY(launch_surface(X, X + 3 * N, X + 6 * N, 1, P, pl->wsin.ptr, rec, s));
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  return BIE_OK;
}

static int drop_stats(const double* rec, long long N, const double* c, double* vol, double* bnd, cudaStream_t s) {
  DevBuf<double> o;
  BIE_TRY(o.alloc(128));
  BIE_TRY(launch_drop_stats(rec, N, c, o.ptr, s));
  std::vector<double> h(128);
  BIE_CUDA_TRY(cudaMemcpyAsync(h.data(), o.ptr, 128 * sizeof(double), cudaMemcpyDeviceToHost, s));
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  double v = 0, m = 0;
  for (int b = 0; b < 64; ++b) {
    v += h[2 * b];
    m = std::max(m, h[2 * b + 1]);
  }
  *vol = v / 3.0;
  *bnd = m;
  return BIE_OK;
}

static int setup_near(bie_ctx* ctx, bie_geom* g, cudaStream_t s);

// Autotuner of the FP32 pair kernel: for large work lists, time the variants (targets per thread 1,
// 2, 4; packed lane pairs for 2 and 4; with or without pipelined source staging) once on this
// geometry's work list (double layer, zero densities: the cost does not depend on the values) and
// keep the fastest.
static int autotune_interdrop(bie_ctx* ctx, bie_geom* g, cudaStream_t s) {
  const long long pairs = g->info.far_pairs + g->info.up_pairs;
  g->info.interdrop_tpt = g->tpt32;
  if (pairs < 500000000LL || g->nblk == 0) return BIE_OK;
  // a geometry of the same drops whose pair count is within 10% of one tuned before in this context
  // (the next time step's geometry, say) reuses that choice
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (const auto& t : ctx->tuned)
      if (t.p == g->p && t.pq == g->pq && t.up == ctx->cfg.upsample && std::llabs(pairs - t.pairs) * 10 <= t.pairs) {
        g->tpt32 = t.tpt;
        g->info.interdrop_tpt = t.tpt;
        return BIE_OK;
      }
  }
  BIE_TRY(g->sQ32.alloc(3 * g->ntarget));
  BIE_TRY(g->uQ32.alloc(3 * g->nup_total));
  BIE_CUDA_TRY(cudaMemsetAsync(g->sQ32.ptr, 0, 3 * g->ntarget * sizeof(float), s));
  BIE_CUDA_TRY(cudaMemsetAsync(g->uQ32.ptr, 0, 3 * g->nup_total * sizeof(float), s));
  cudaEvent_t e0, e1;
  BIE_CUDA_TRY(cudaEventCreate(&e0));
  BIE_CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  // targets per thread 1 (scalar FP32), 2 and 4 (packed lane pairs), 12, 14 (packed, with the next
  // chunk of sources loaded while the current one is summed), 24, 34 (4 targets, 32-source chunks)
  const int cand[7] = {1, 2, 4, 12, 14, 24, 34};
  // time a leading part of the work list of about 5e10 pairs (at least 32 blocks per SM); blocks carry
  // similar work, so its ranking is the full list's
  const int nsample = (int)std::min<long long>(
      g->nblk, std::max<long long>(32LL * ctx->sms, (long long)((double)g->nblk * std::min(1.0, 5e10 / (double)pairs))));
  for (int ci = 0; ci < 7; ++ci) {
    cudaEventRecord(e0, s);
    int st = launch_interdrop<float>(1, cand[ci], nsample, g->items.ptr, g->blk_item.ptr, g->tile_t0.ptr,
                                     g->tile_n.ptr, g->tile_drop.ptr, g->tgt_loc.ptr, g->toff.ptr, g->ngd.ptr,
                                     g->rec_std.ptr, g->centre_d.ptr, g->sX32.ptr, g->sN32.ptr, g->sQ32.ptr,
                                     g->ntarget, g->uX32.ptr, g->uN32.ptr, g->uQ32.ptr, g->nup_total, g->wD_all.ptr,
                                     g->partial.ptr, s);
    cudaEventRecord(e1, s);
    if (st != BIE_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return st;
    }
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      g->tpt32 = cand[ci];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g->info.interdrop_tpt = g->tpt32;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->tuned.size() >= 16) ctx->tuned.erase(ctx->tuned.begin());
  ctx->tuned.push_back({g->p, g->pq, ctx->cfg.upsample, pairs, g->tpt32});
  return BIE_OK;
}

static int setup_interdrop(bie_ctx* ctx, bie_geom* g, cudaStream_t s) {
  const int nd = g->ndrop;
  const int U = ctx->cfg.upsample;
  // centres from the degree-0 coefficients: x_0^0 = sqrt(4 pi) c
  std::vector<double> xc(g->ncoef_total);
  BIE_CUDA_TRY(cudaMemcpy(xc.data(), g->xcoef.ptr, xc.size() * sizeof(double), cudaMemcpyDeviceToHost));
  g->centre.assign(3 * nd, 0.0);
  g->bound.assign(nd, 0.0);
  g->hdrop.assign(nd, 0.0);
  g->volume.assign(nd, 0.0);
  g->up_off.assign(nd, 0);
  g->up_n.assign(nd, 0);
  g->up_P.assign(nd, 0);
  long long uo = 0;
  for (int d = 0; d < nd; ++d) {
    for (int c = 0; c < 3; ++c) g->centre[3 * d + c] = xc[g->coef_off[d] + c * ncoef(g->p[d])] / std::sqrt(4 * kPi);
    g->up_P[d] = U * (g->p[d] + 1) - 1;
    g->up_off[d] = uo;
    g->up_n[d] = ngrid(g->up_P[d]);
    uo += g->up_n[d];
  }
  g->nup_total = uo;
  BIE_TRY(g->rec_up.alloc(7 * uo));
  BIE_TRY(g->centre_d.upload(g->centre));
  // set-up stages are timed as phases when profiling is on
  std::unique_ptr<Phase> stage(new Phase(ctx, "setup_records", s));
  for (int d = 0; d < nd; ++d) {
    const int p = g->p[d];
    // volume by the regular rule on the grid of degree 2p+1, mean radius, h = R pi/(p+1)
    const int P2 = 2 * p + 1;
    DevBuf<double> rec2;
    BIE_TRY(rec2.alloc(7 * ngrid(P2)));
    BIE_TRY(drop_records(ctx, g, d, P2, rec2.ptr, s));
    double vol, dummy;
    BIE_TRY(drop_stats(rec2.ptr, ngrid(P2), &g->centre[3 * d], &vol, &dummy, s));
    g->volume[d] = vol;
    const double R = std::cbrt(3.0 * vol / (4.0 * kPi));
    g->hdrop[d] = R * kPi / (p + 1);
    // upsampled grid records and the bounding radius about the centre
    double* ru = g->rec_up.ptr + 7 * g->up_off[d];
    BIE_TRY(drop_records(ctx, g, d, g->up_P[d], ru, s));
    double v2;
    BIE_TRY(drop_stats(ru, g->up_n[d], &g->centre[3 * d], &v2, &g->bound[d], s));
  }
  // per-target bookkeeping
  stage.reset(new Phase(ctx, "setup_sources", s));
  const long long nt = g->ntarget;
  std::vector<int> tdrop(nt), ngd(nd);
  std::vector<long long> tloc(nt), voff(nd);
  for (int d = 0; d < nd; ++d) {
    ngd[d] = (int)ngrid(g->p[d]);
    voff[d] = 3 * g->tgt_off[d];
    for (long long l = 0; l < ngd[d]; ++l) {
      tdrop[g->tgt_off[d] + l] = d;
      tloc[g->tgt_off[d] + l] = l;
    }
  }
  BIE_TRY(g->tdrop.upload(tdrop));
  BIE_TRY(g->tgt_loc.upload(tloc));
  BIE_TRY(g->toff.upload(g->tgt_off));
  BIE_TRY(g->ngd.upload(ngd));
  BIE_TRY(g->val_off_all.upload(voff));
  // source geometry relative to the drop centres, FP64 and FP32
  const long long ns = nt;
  BIE_TRY(g->sX64.alloc(3 * ns));
  BIE_TRY(g->sN64.alloc(3 * ns));
  BIE_TRY(g->sX32.alloc(3 * ns));
  BIE_TRY(g->sN32.alloc(3 * ns));
  BIE_TRY(g->uX64.alloc(3 * uo));
  BIE_TRY(g->uN64.alloc(3 * uo));
  BIE_TRY(g->uX32.alloc(3 * uo));
  BIE_TRY(g->uN32.alloc(3 * uo));
  for (int d = 0; d < nd; ++d) {
    const double* c = &g->centre[3 * d];
    const double* rs = g->rec_std.ptr + 7 * g->tgt_off[d];
    const double* ru = g->rec_up.ptr + 7 * g->up_off[d];
    BIE_TRY(launch_source_geometry<double>(rs, ngd[d], c, g->sX64.ptr + g->tgt_off[d], g->sN64.ptr + g->tgt_off[d],
                                           ns, s));
    BIE_TRY(launch_source_geometry<float>(rs, ngd[d], c, g->sX32.ptr + g->tgt_off[d], g->sN32.ptr + g->tgt_off[d],
                                          ns, s));
    BIE_TRY(launch_source_geometry<double>(ru, g->up_n[d], c, g->uX64.ptr + g->up_off[d],
                                           g->uN64.ptr + g->up_off[d], uo, s));
    BIE_TRY(launch_source_geometry<float>(ru, g->up_n[d], c, g->uX32.ptr + g->up_off[d], g->uN32.ptr + g->up_off[d],
                                          uo, s));
  }
  // region classification on the device, per-(tile, drop) masks on the device, work list on the host
  stage.reset(new Phase(ctx, "setup_classify", s));
  std::vector<long long> tile_t0;
  std::vector<int> tile_n, tile_drop;
  for (int d = 0; d < nd; ++d)
    for (long long l = 0; l < ngd[d]; l += kTile) {
      tile_t0.push_back(g->tgt_off[d] + l);
      tile_n.push_back((int)std::min<long long>(kTile, ngd[d] - l));
      tile_drop.push_back(d);
    }
  const int ntile = (int)tile_t0.size();
  BIE_TRY(g->tile_t0.upload(tile_t0));
  BIE_TRY(g->tile_n.upload(tile_n));
  std::vector<TileMask> tmask((size_t)ntile * nd);
  {
    DevBuf<unsigned char> reg;
    DevBuf<double> bnd, hh;
    DevBuf<long long> uoff, un;
    DevBuf<TileMask> tm;
    BIE_TRY(reg.alloc((size_t)nt * nd));
    BIE_TRY(bnd.upload(g->bound));
    BIE_TRY(hh.upload(g->hdrop));
    BIE_TRY(uoff.upload(g->up_off));
    BIE_TRY(un.upload(g->up_n));
    BIE_TRY(tm.alloc(tmask.size()));
    BIE_TRY(launch_classify(g->rec_std.ptr, nt, g->tdrop.ptr, g->tgt_loc.ptr, g->toff.ptr, g->ngd.ptr, nd,
                            g->centre_d.ptr, bnd.ptr, hh.ptr, ctx->cfg.a_tilde, g->rec_up.ptr, uoff.ptr, un.ptr,
                            reg.ptr, s));
    BIE_TRY(launch_tile_masks(reg.ptr, nd, g->tile_t0.ptr, g->tile_n.ptr, ntile, tm.ptr, s));
    BIE_CUDA_TRY(cudaStreamSynchronize(s));
    stage.reset(new Phase(ctx, "setup_masks_copy", s));
    BIE_CUDA_TRY(cudaMemcpyAsync(tmask.data(), tm.ptr, tmask.size() * sizeof(TileMask), cudaMemcpyDeviceToHost, s));
    BIE_CUDA_TRY(cudaStreamSynchronize(s));
  }
  stage.reset(new Phase(ctx, "setup_worklist", s));
  auto popc = [](const unsigned* m) {
    int c = 0;
    for (int q = 0; q < 4; ++q) c += __builtin_popcount(m[q]);
    return c;
  };
  // total sources over all tiles, to aim at >= 8 blocks per SM overall
  long long all_sources = 0;
  for (int ti = 0; ti < ntile; ++ti)
    for (int j = 0; j < nd; ++j) {
      if (j == tile_drop[ti]) continue;
      const TileMask& tmj = tmask[(size_t)ti * nd + j];
      all_sources += (popc(tmj.m[0]) ? ngd[j] : 0) + (popc(tmj.m[1]) ? g->up_n[j] : 0);
    }
  const long long cap_global = std::max<long long>(2048, std::min<long long>(65536, all_sources / (8LL * ctx->sms)));
  std::vector<PairItem> items;
  std::vector<int> blk_item, tile_blk(ntile + 1, 0);
  long long far_pairs = 0, up_pairs = 0, slots = 0;
  g->near.clear();
  for (int ti = 0; ti < ntile; ++ti) {
    std::vector<PairItem> mine;
    long long total = 0;
    for (int j = 0; j < nd; ++j) {
      if (j == tile_drop[ti]) continue;
      PairItem a{}, b{};
      const TileMask& tmj = tmask[(size_t)ti * nd + j];
      if (tmj.inside) {
        set_error("drops overlap: a grid point of drop " + std::to_string(tile_drop[ti]) + " lies inside drop " +
                  std::to_string(j));
        return BIE_EOVERLAP;
      }
      for (int q = 0; q < 4; ++q) {
        a.mask[q] = tmj.m[0][q];
        b.mask[q] = tmj.m[1][q];
      }
      const int n0 = popc(tmj.m[0]), n1 = popc(tmj.m[1]);
      if (tmj.m[2][0] | tmj.m[2][1] | tmj.m[2][2] | tmj.m[2][3])
        for (int k = 0; k < tile_n[ti]; ++k)
          if ((tmj.m[2][k >> 5] >> (k & 31)) & 1u) g->near.emplace_back(tile_t0[ti] + k, j);
      if (n0) {
        a.tile = ti;
        a.src_drop = j;
        a.grid = 0;
        a.s0 = g->tgt_off[j];
        a.s1 = g->tgt_off[j] + ngd[j];
        mine.push_back(a);
        total += ngd[j];
        far_pairs += (long long)n0 * ngd[j];
        slots += (long long)kTile * ngd[j];
      }
      if (n1) {
        b.tile = ti;
        b.src_drop = j;
        b.grid = 1;
        b.s0 = g->up_off[j];
        b.s1 = g->up_off[j] + g->up_n[j];
        mine.push_back(b);
        total += g->up_n[j];
        up_pairs += (long long)n1 * g->up_n[j];
        slots += (long long)kTile * g->up_n[j];
      }
    }
    // split the tile's items into blocks of at most `cap` sources
    const long long cap = std::max(cap_global, (total + 15) / 16);  // at most 16 blocks per tile
    tile_blk[ti] = (int)blk_item.size();
    long long used = cap;  // forces a new block at the first item
    for (auto it : mine) {
      long long s0 = it.s0;
      while (s0 < it.s1) {
        if (used >= cap) {
          blk_item.push_back((int)items.size());
          used = 0;
        }
        const long long take = std::min(it.s1 - s0, cap - used);
        PairItem piece = it;
        piece.s0 = s0;
        piece.s1 = s0 + take;
        items.push_back(piece);
        used += take;
        s0 += take;
      }
    }
  }
  tile_blk[ntile] = (int)blk_item.size();
  stage.reset(new Phase(ctx, "setup_worklist_upload", s));
  const int nblk = (int)blk_item.size();
  blk_item.push_back((int)items.size());
  g->ntile = ntile;
  g->nblk = nblk;
  if (!items.empty()) BIE_TRY(g->items.upload(items));
  BIE_TRY(g->blk_item.upload(blk_item));
  BIE_TRY(g->tile_blk.upload(tile_blk));
  BIE_TRY(g->tile_drop.upload(tile_drop));
  BIE_TRY(g->partial.alloc((size_t)std::max(1, nblk) * 3 * kTile));
  std::vector<double> wS(nd), wD(nd), wSr(nd), wDr(nd);
  for (int d = 0; d < nd; ++d) {
    wS[d] = -1.0 / (4 * kPi);
    wD[d] = (g->lambda[d] - 1.0) / (4 * kPi);
    wSr[d] = 1.0 / (8 * kPi);
    wDr[d] = 1.0 / (4 * kPi);
  }
  BIE_TRY(g->wS_all.upload(wS));
  BIE_TRY(g->wD_all.upload(wD));
  BIE_TRY(g->wSr_all.upload(wSr));
  BIE_TRY(g->wDr_all.upload(wDr));
  g->info.far_pairs = far_pairs;
  g->info.up_pairs = up_pairs;
  g->info.pair_slots = slots;
  g->info.near_targets = (long long)g->near.size();
  BIE_TRY(g->up_off_d.upload(g->up_off));
  BIE_TRY(g->up_n_d.upload(g->up_n));
  stage.reset(new Phase(ctx, "setup_autotune", s));
  BIE_TRY(autotune_interdrop(ctx, g, s));
  stage.reset();
  for (auto& G : g->groups) {
    std::vector<long long> so, uo2;
    for (int d : G->drops) {
      so.push_back(g->tgt_off[d]);
      uo2.push_back(g->up_off[d]);
    }
    BIE_TRY(G->src_off_std.upload(so));
    BIE_TRY(G->src_off_up.upload(uo2));
  }
  if (!g->near.empty()) {
    Phase ph(ctx, "setup_near", s);
    BIE_TRY(setup_near(ctx, g, s));
  }
  g->interdrop_ready = true;
  return BIE_OK;
}

// Source densities of every drop on its standard and upsampled grids, weighted by the regular
// quadrature weight and area density (Sec. 2.1, Sec. 2.3).
template <typename R>
static int source_densities(bie_geom* g, const double* dens, R* Qs, R* Qu, cudaStream_t s) {
  bie_ctx* ctx = g->ctx;
  Phase ph(ctx, "source_synth", s);
  for (auto& Gp : g->groups) {
    auto& G = *Gp;
    const int p = G.p;
    const int Pu = ctx->cfg.upsample * (p + 1) - 1;
    const long long nd = (long long)G.drops.size();
    const long long need = nd * 3 * ((long long)(p + 1) * (Pu + 1) * 2 + ngrid(Pu));
    R* H;
    if (sizeof(R) == 8) {
      BIE_TRY(g->syn64.alloc(need));
      H = reinterpret_cast<R*>(g->syn64.ptr);
    } else {
      BIE_TRY(g->syn32.alloc(need));
      H = reinterpret_cast<R*>(g->syn32.ptr);
    }
    for (int gridk = 0; gridk < 2; ++gridk) {
      const int P = gridk ? Pu : p;
      const long long N = ngrid(P);
      Plan* pl;
      BIE_TRY(get_plan(ctx, p, P, &pl));
      R* grid = H + nd * 3 * (long long)(p + 1) * (P + 1) * 2;
      BIE_TRY((launch_leg_synth<double, R>(dens, G.foff3.ptr, 0, nd * 3, p, pl->T0_<R>(), P + 1, H, 0, s)));
      BIE_TRY((launch_phi_synth<R, R>(H, nd * 3, p, P, pl->cs_<R>(), grid, nullptr, N, s)));
      if (gridk == 0)
        BIE_TRY(launch_weight_sources<R>(grid, g->rec_std.ptr, G.src_off_std.ptr, N, nd, Qs, g->ntarget, s));
      else
        BIE_TRY(launch_weight_sources<R>(grid, g->rec_up.ptr, G.src_off_up.ptr, N, nd, Qu, g->nup_total, s));
    }
  }
  return BIE_OK;
}

// Closest points x* of near pairs (Sec. 2.3): damped Newton in a rotated frame that puts the seed
// (the source drop's standard-grid point nearest to x0) on the equator; then the check points
// x_l = x* + h_j sqrt(l) e, e = (x0 - x*)/|x0 - x*|, l = 1..L, and the grid (standard or upsampled)
// each is summed on.  x0: 3 per pair (host); seeds: standard-grid index per pair.  Fills d0 and the
// parameters of x* in drop j's own frame into the pairs and returns the check points [pair][L][3]
// and their grids [pair][L] on the device.
static int near_points(bie_ctx* ctx, bie_geom* g, std::vector<NearPair>& pairs, const std::vector<double>& x0,
                       const std::vector<int>& hseed, DevBuf<double>& pts_d, DevBuf<int>& grid_d, cudaStream_t s) {
  const int npair = (int)pairs.size();
  const int L = ctx->cfg.n_interp;
  DevBuf<NearPair> dpairs;
  BIE_TRY(dpairs.upload(pairs));
  // rotated shape coefficients: (alpha, beta) = (phi_b, theta_a - pi/2) puts the seed (latitude a,
  // longitude b) at the equator.  The phases e^{i m alpha} of every pair are applied in one launch;
  // then the pairs of one degree and one seed latitude share one rotation launch (the small-d blocks
  // of that beta), and one Newton launch serves every pair.  The rotated coefficients lie in group
  // order, [pair][3][(p+1)^2].
  std::unique_ptr<Phase> stage(new Phase(ctx, "near_newton", s));
  std::vector<double> alpha(npair), beta(npair), hres(5 * (size_t)npair);
  std::map<std::pair<int, int>, std::vector<int>> groups;  // (degree, seed latitude) -> pairs
  int pmax = 0;
  for (int i = 0; i < npair; ++i) {
    const int p = g->p[pairs[i].src_drop];
    pmax = std::max(pmax, p);
    groups[{p, hseed[i] / (2 * p + 2)}].push_back(i);
  }
  struct RotGroup {
    int p, n;
    long long base, fo_at, blk_at, blk_n;
  };
  std::vector<RotGroup> rg;
  std::vector<long long> xr_off(npair), fo_all;
  std::vector<double> blocks_all, ph(2 * (size_t)npair * (pmax + 1), 0.0);
  long long xo = 0;
  for (const auto& kv : groups) {
    const int p = kv.first.first, a = kv.first.second;
    const std::vector<int>& idx = kv.second;
    const int nb = 2 * p + 2;
    const long long nc = ncoef(p);
    std::vector<double> t, w;
    gauss_legendre(p + 1, t, w);
    const double be = std::acos(t[a]) - 0.5 * kPi;
    std::vector<double> blk(wigner_block_stride(p));
    wigner_blocks(p, be, blk.data());
    rg.push_back({p, (int)idx.size(), xo, (long long)fo_all.size(), (long long)blocks_all.size(), (long long)blk.size()});
    blocks_all.insert(blocks_all.end(), blk.begin(), blk.end());
    for (size_t k = 0; k < idx.size(); ++k) {
      const int i = idx[k];
      alpha[i] = kPi * (hseed[i] % nb) / (p + 1);
      beta[i] = be;
      xr_off[i] = xo + (long long)k * 3 * nc;
      for (int c = 0; c < 3; ++c) fo_all.push_back(xr_off[i] + c * nc);
      for (int m = 0; m <= p; ++m) {
        ph[2 * ((size_t)i * (pmax + 1) + m)] = std::cos(m * alpha[i]);
        ph[2 * ((size_t)i * (pmax + 1) + m) + 1] = std::sin(m * alpha[i]);
      }
    }
    xo += (long long)idx.size() * 3 * nc;
  }
  std::vector<int> pd(g->p.begin(), g->p.end());
  DevBuf<int> pdeg;
  DevBuf<double> shifted, xr, dblk, dph, dx0, res;
  DevBuf<long long> dfo, dxo, dcoef_off;
  BIE_TRY(pdeg.upload(pd));
  BIE_TRY(dcoef_off.upload(g->coef_off));
  BIE_TRY(dph.upload(ph));
  BIE_TRY(dxo.upload(xr_off));
  BIE_TRY(dfo.upload(fo_all));
  BIE_TRY(dblk.upload(blocks_all));
  BIE_TRY(dx0.upload(x0));
  BIE_TRY(shifted.alloc(xo));
  BIE_TRY(xr.alloc(xo));
  BIE_TRY(res.alloc(5 * (size_t)npair));
  BIE_TRY(launch_near_phase_shift(dpairs.ptr, npair, g->xcoef.ptr, dcoef_off.ptr, pdeg.ptr, pmax, dph.ptr, dxo.ptr,
                                  shifted.ptr, s));
  for (const auto& G : rg) {
    const long long nc = ncoef(G.p);
    BIE_TRY((launch_rotate<double, double>(shifted.ptr, dfo.ptr + G.fo_at, 3, G.n, G.p, dblk.ptr + G.blk_at, G.blk_n,
                                           1, 1, (const double*)nullptr, xr.ptr + G.base, 3 * nc, s)));
  }
  DevBuf<double> rtab;
  BIE_TRY(rtab.alloc(near_rec_table_doubles(pmax)));
  BIE_TRY(launch_near_rec_table(pmax, rtab.ptr, s));
  BIE_TRY(launch_near_newton(dpairs.ptr, npair, xr.ptr, pdeg.ptr, dxo.ptr, dx0.ptr, rtab.ptr, res.ptr, s));
  BIE_CUDA_TRY(cudaMemcpyAsync(hres.data(), res.ptr, hres.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  stage.reset(new Phase(ctx, "near_checkpoints", s));
  std::vector<double> pts(3 * (size_t)npair * L);
  for (int i = 0; i < npair; ++i) {
    const int j = pairs[i].src_drop;
    const double th = hres[5 * i], phv = hres[5 * i + 1];
    const double xs[3] = {hres[5 * i + 2], hres[5 * i + 3], hres[5 * i + 4]};
    double e[3], d0 = 0;
    for (int c = 0; c < 3; ++c) {
      e[c] = x0[3 * i + c] - xs[c];
      d0 += e[c] * e[c];
    }
    d0 = std::sqrt(d0);
    for (int c = 0; c < 3; ++c) e[c] /= d0;
    pairs[i].d0 = d0;
    // parameters of x* in drop j's own frame: v = R_z(alpha) R_y(beta) s(theta*, phi*)
    const double sv[3] = {std::sin(th) * std::cos(phv), std::sin(th) * std::sin(phv), std::cos(th)};
    const double cb = std::cos(beta[i]), sb = std::sin(beta[i]), ca = std::cos(alpha[i]), sa = std::sin(alpha[i]);
    const double y0 = cb * sv[0] + sb * sv[2], y1 = sv[1], y2 = -sb * sv[0] + cb * sv[2];
    const double v0 = ca * y0 - sa * y1, v1 = sa * y0 + ca * y1, v2 = y2;
    pairs[i].theta_v = std::acos(std::max(-1.0, std::min(1.0, v2)));
    pairs[i].phi_v = std::atan2(v1, v0);
    for (int l = 1; l <= L; ++l)
      for (int c = 0; c < 3; ++c) pts[3 * ((size_t)i * L + (l - 1)) + c] = xs[c] + g->hdrop[j] * std::sqrt((double)l) * e[c];
  }
  BIE_TRY(pts_d.upload(pts));
  BIE_TRY(grid_d.alloc((size_t)npair * L));
  DevBuf<double> bnd, hh;
  DevBuf<long long> uoff, un;
  BIE_TRY(bnd.upload(g->bound));
  BIE_TRY(hh.upload(g->hdrop));
  BIE_TRY(uoff.upload(g->up_off));
  BIE_TRY(un.upload(g->up_n));
  BIE_TRY(launch_near_checkgrid(dpairs.ptr, npair, L, pts_d.ptr, g->centre_d.ptr, bnd.ptr, hh.ptr, ctx->cfg.a_tilde,
                                g->rec_up.ptr, uoff.ptr, un.ptr, grid_d.ptr, s));
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  return BIE_OK;
}

// Device tables the near-singular interpolation reads (degrees, h, coefficient offsets) and the
// buffers of the on-surface expansions, made once per geometry.
static int near_tables(bie_geom* g) {
  if (g->pdeg_d.ptr) return BIE_OK;
  BIE_TRY(g->selfvals.alloc(3 * g->ntarget));
  BIE_TRY(g->selfcoef.alloc(g->ncoef_total));
  BIE_TRY(g->hdrop_d.upload(g->hdrop));
  BIE_TRY(g->coef_off_d.upload(g->coef_off));
  std::vector<int> pd(g->p.begin(), g->p.end());
  BIE_TRY(g->pdeg_d.upload(pd));
  return BIE_OK;
}

// Near-singular set-up (Sec. 2.3) for the drops' own targets: seeds on the device, then near_points.
static int setup_near(bie_ctx* ctx, bie_geom* g, cudaStream_t s) {
  auto& nr = g->near;
  std::sort(nr.begin(), nr.end());
  const int npair = (int)nr.size();
  const int L = ctx->cfg.n_interp;
  std::vector<NearPair> pairs(npair);
  std::vector<int> tbeg;
  for (int i = 0; i < npair; ++i) {
    pairs[i].target = nr[i].first;
    pairs[i].src_drop = nr[i].second;
    if (i == 0 || nr[i].first != nr[i - 1].first) tbeg.push_back(i);
  }
  g->nnear_tgt = (int)tbeg.size();
  tbeg.push_back(npair);
  BIE_TRY(g->npairs.upload(pairs));
  BIE_TRY(g->ntbeg.upload(tbeg));
  DevBuf<int> seed;
  BIE_TRY(seed.alloc(npair));
  BIE_TRY(launch_near_seed(g->npairs.ptr, npair, g->rec_std.ptr, g->toff.ptr, g->ngd.ptr, g->tgt_loc.ptr,
                           g->tdrop.ptr, seed.ptr, s));
  std::vector<int> hseed(npair);
  BIE_CUDA_TRY(cudaMemcpyAsync(hseed.data(), seed.ptr, npair * sizeof(int), cudaMemcpyDeviceToHost, s));
  std::vector<double> rec(7 * g->ntarget);
  BIE_CUDA_TRY(cudaMemcpyAsync(rec.data(), g->rec_std.ptr, rec.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<double> x0(3 * npair);
  for (int i = 0; i < npair; ++i) {
    const long long tt = pairs[i].target;
    int di = 0;
    while (di + 1 < g->ndrop && g->tgt_off[di + 1] <= tt) ++di;
    const long long ngi = ngrid(g->p[di]), l = tt - g->tgt_off[di];
    for (int c = 0; c < 3; ++c) x0[3 * i + c] = rec[7 * g->tgt_off[di] + c * ngi + l];
  }
  BIE_TRY(near_points(ctx, g, pairs, x0, hseed, g->npts, g->ngrid_l, s));
  BIE_TRY(g->npairs.upload(pairs));
  BIE_TRY(g->ncv.alloc(3 * (size_t)npair * L));
  BIE_TRY(near_tables(g));
  long long npairs_eval = 0;
  std::vector<int> hgrid((size_t)npair * L);
  BIE_CUDA_TRY(cudaMemcpy(hgrid.data(), g->ngrid_l.ptr, hgrid.size() * sizeof(int), cudaMemcpyDeviceToHost));
  for (int i = 0; i < npair; ++i)
    for (int l = 0; l < L; ++l) {
      const int j = pairs[i].src_drop;
      npairs_eval += hgrid[(size_t)i * L + l] ? g->up_n[j] : ngrid(g->p[j]);
    }
  g->info.near_pairs = npairs_eval;
  return BIE_OK;
}

// Self-interaction values of every drop as SH coefficients (weighted units): the on-surface
// values of the near-singular interpolation come from these expansions.
static int near_snapshot(bie_geom* g, cudaStream_t s) {
  BIE_CUDA_TRY(cudaMemcpyAsync(g->selfvals.ptr, g->vals.ptr, 3 * g->ntarget * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
  BIE_TRY(analyze_groups(g->ctx, g, g->selfvals.ptr, g->selfcoef.ptr, s));
  return BIE_OK;
}

static int near_apply(bie_geom* g, int kind, bool raw, int prec, const double* dens, cudaStream_t s) {
  if (g->near.empty()) return BIE_OK;
  bie_ctx* ctx = g->ctx;
  const int npair = (int)g->near.size(), L = ctx->cfg.n_interp;
  const double* wts = kind == 0 ? (raw ? g->wSr_all.ptr : g->wS_all.ptr) : (raw ? g->wDr_all.ptr : g->wD_all.ptr);
  // The check-point values are always summed in FP64: the interpolation through (0, h sqrt(l)),
  // l = 1..8, amplifies their errors by its Lebesgue constant (about 1.9e3 on [0, h]).
  if (prec != BIE_FP64) {
    BIE_TRY(g->sQ64.alloc(3 * g->ntarget));
    BIE_TRY(g->uQ64.alloc(3 * g->nup_total));
    BIE_TRY(source_densities<double>(g, dens, g->sQ64.ptr, g->uQ64.ptr, s));
  }
  Phase ph(ctx, "near", s);
  BIE_TRY(launch_near_checks<double>(kind, g->npairs.ptr, npair, L, g->npts.ptr, g->ngrid_l.ptr, g->centre_d.ptr,
                                     g->toff.ptr, g->ngd.ptr, g->up_off_d.ptr, g->up_n_d.ptr, g->sX64.ptr, g->sN64.ptr,
                                     g->sQ64.ptr, g->ntarget, g->uX64.ptr, g->uN64.ptr, g->uQ64.ptr, g->nup_total,
                                     wts, g->ncv.ptr, s));
  return launch_near_interp(g->npairs.ptr, g->ntbeg.ptr, g->nnear_tgt, L, kind, g->selfcoef.ptr, dens,
                            g->coef_off_d.ptr, g->pdeg_d.ptr, g->hdrop_d.ptr, wts, g->ncv.ptr, g->tdrop.ptr,
                            g->tgt_loc.ptr, g->val_off_all.ptr, g->ngd.ptr, g->vals.ptr, s);
}

template <typename R>
static int interdrop_apply(bie_geom* g, int kind, bool raw, const double* dens, cudaStream_t s, bool df) {
  bie_ctx* ctx = g->ctx;
  R *Qs, *Qu;
  const R *Xs, *Ns, *Xu, *Nu;
  if (sizeof(R) == 8) {
    BIE_TRY(g->sQ64.alloc(3 * g->ntarget));
    BIE_TRY(g->uQ64.alloc(3 * g->nup_total));
    Qs = reinterpret_cast<R*>(g->sQ64.ptr);
    Qu = reinterpret_cast<R*>(g->uQ64.ptr);
    Xs = reinterpret_cast<const R*>(g->sX64.ptr);
    Ns = reinterpret_cast<const R*>(g->sN64.ptr);
    Xu = reinterpret_cast<const R*>(g->uX64.ptr);
    Nu = reinterpret_cast<const R*>(g->uN64.ptr);
  } else {
    BIE_TRY(g->sQ32.alloc(3 * g->ntarget));
    BIE_TRY(g->uQ32.alloc(3 * g->nup_total));
    Qs = reinterpret_cast<R*>(g->sQ32.ptr);
    Qu = reinterpret_cast<R*>(g->uQ32.ptr);
    Xs = reinterpret_cast<const R*>(g->sX32.ptr);
    Ns = reinterpret_cast<const R*>(g->sN32.ptr);
    Xu = reinterpret_cast<const R*>(g->uX32.ptr);
    Nu = reinterpret_cast<const R*>(g->uN32.ptr);
  }
  BIE_TRY(source_densities<R>(g, dens, Qs, Qu, s));
  const double* wts = kind == 0 ? (raw ? g->wSr_all.ptr : g->wS_all.ptr) : (raw ? g->wDr_all.ptr : g->wD_all.ptr);
  if (df) {
    Phase ph(ctx, "interdrop_df", s);
    BIE_TRY(launch_interdrop_df(kind, g->nblk, g->items.ptr, g->blk_item.ptr, g->tile_t0.ptr, g->tile_n.ptr,
                                g->tile_drop.ptr, g->tgt_loc.ptr, g->toff.ptr, g->ngd.ptr, g->rec_std.ptr,
                                g->centre_d.ptr, g->sX64.ptr, g->sN64.ptr, g->sQ64.ptr, g->ntarget, g->uX64.ptr,
                                g->uN64.ptr, g->uQ64.ptr, g->nup_total, wts, g->partial.ptr, s));
  } else {
    Phase ph(ctx, sizeof(R) == 8 ? "interdrop_f64" : "interdrop_f32", s);
    BIE_TRY(launch_interdrop<R>(kind, sizeof(R) == 8 ? g->tpt64 : g->tpt32, g->nblk, g->items.ptr, g->blk_item.ptr, g->tile_t0.ptr, g->tile_n.ptr,
                                g->tile_drop.ptr, g->tgt_loc.ptr, g->toff.ptr, g->ngd.ptr, g->rec_std.ptr,
                                g->centre_d.ptr, Xs, Ns, Qs, g->ntarget, Xu, Nu, Qu, g->nup_total, wts,
                                g->partial.ptr, s));
  }
  Phase ph(ctx, "interdrop_reduce", s);
  return launch_reduce_tiles(g->partial.ptr, g->tile_blk.ptr, g->tile_t0.ptr, g->tile_n.ptr, g->tile_drop.ptr,
                             g->tgt_loc.ptr, g->val_off_all.ptr, g->ngd.ptr, g->ntile, g->vals.ptr, s);
}

// ---- layer potentials at points off the surfaces (Sec. 1, with the region rules of Sec. 2.1-2.3) ----
// The points go through the machinery of the drops' own targets: each chunk of points becomes a
// set of 128-point tiles with a record layout like a drop's (one pseudo-drop per tile, numbered
// after the real drops, whose centre is the tile's mean point), the region masks of every (tile,
// drop) pair make a work list for the pair kernels, and the Omega_2 pairs take the near-singular
// interpolation anchored at the exterior limit of the source drop's on-surface values.
constexpr long long kPtChunk = 32768;  // points per pass at most: 256 tiles

static int eval_layers(bie_ctx* ctx, bie_geom* g, long long npt, const double* pts, const double* const dens[2],
                       double* const out[2], int precision, cudaStream_t s) {
  const bool raw = (precision & BIE_RAW) != 0;
  const int prec = precision & 0xff;
  if ((precision & ~(0xff | BIE_RAW)) != 0 || (prec != BIE_FP64 && prec != BIE_MIXED && prec != BIE_DF)) {
    set_error("precision must be BIE_FP64, BIE_MIXED or BIE_DF, optionally | BIE_RAW");
    return BIE_EINVAL;
  }
  if (npt < 0 || npt > 0x7fffffffLL) {
    set_error("npoint must lie in [0, 2^31)");
    return BIE_EINVAL;
  }
  if (npt == 0) return BIE_OK;
  std::vector<int> kinds;  // the layers asked for: 0 single, 1 double
  for (int k = 0; k < 2; ++k)
    if (out[k]) {
      kinds.push_back(k);
      BIE_CUDA_TRY(cudaMemsetAsync(out[k], 0, 3 * npt * sizeof(double), s));
    }
  if (!g->interdrop_ready) BIE_TRY(setup_interdrop(ctx, g, s));
  const int nd = g->ndrop;
  // points per pass: kPtChunk, fewer when there are so many drops that the per-(point, drop) scratch
  // of the classification would pass 2^26 entries
  const long long chunk =
      std::max<long long>(kTile, std::min<long long>(kPtChunk, ((1LL << 26) / nd) / kTile * kTile));
  auto weights = [&](int kind) {
    return kind == 0 ? (raw ? g->wSr_all.ptr : g->wS_all.ptr) : (raw ? g->wDr_all.ptr : g->wD_all.ptr);
  };
  // source densities of each layer, in the precision of its pair sums
  DevBuf<float> q32[2][2];
  DevBuf<double> q64[2][2];
  for (int k : kinds) {
    if (prec == BIE_MIXED) {
      BIE_TRY(q32[k][0].alloc(3 * g->ntarget));
      BIE_TRY(q32[k][1].alloc(3 * g->nup_total));
      BIE_TRY(source_densities<float>(g, dens[k], q32[k][0].ptr, q32[k][1].ptr, s));
    } else {
      BIE_TRY(q64[k][0].alloc(3 * g->ntarget));
      BIE_TRY(q64[k][1].alloc(3 * g->nup_total));
      BIE_TRY(source_densities<double>(g, dens[k], q64[k][0].ptr, q64[k][1].ptr, s));
    }
  }
  // tile-local tables, the same for every chunk
  const int mt = (int)((chunk + kTile - 1) / kTile);
  std::vector<long long> h_t0(mt), h_loc(chunk), h_toff(nd + mt, 0), h_voff(nd + mt, 0);
  std::vector<int> h_drop(mt), h_ngd(nd + mt, 0);
  for (int ti = 0; ti < mt; ++ti) {
    h_t0[ti] = (long long)ti * kTile;
    h_drop[ti] = nd + ti;
    h_toff[nd + ti] = (long long)ti * kTile;
    h_ngd[nd + ti] = kTile;
    h_voff[nd + ti] = (long long)ti * 3 * kTile;
  }
  for (long long k = 0; k < chunk; ++k) h_loc[k] = k % kTile;
  DevBuf<long long> d_t0, d_loc, d_toff, d_voff, d_uoff, d_un;
  DevBuf<int> d_drop, d_ngd, d_n, d_blk_item, d_tile_blk;
  DevBuf<double> d_rec, d_cen, d_vals, d_part, d_bnd, d_h;
  DevBuf<unsigned char> d_region;
  DevBuf<TileMask> d_tm;
  DevBuf<PairItem> d_items;
  BIE_TRY(d_t0.upload(h_t0));
  BIE_TRY(d_loc.upload(h_loc));
  BIE_TRY(d_toff.upload(h_toff));
  BIE_TRY(d_voff.upload(h_voff));
  BIE_TRY(d_drop.upload(h_drop));
  BIE_TRY(d_ngd.upload(h_ngd));
  BIE_TRY(d_bnd.upload(g->bound));
  BIE_TRY(d_h.upload(g->hdrop));
  BIE_TRY(d_uoff.upload(g->up_off));
  BIE_TRY(d_un.upload(g->up_n));
  BIE_TRY(d_rec.alloc((size_t)mt * 7 * kTile));
  BIE_TRY(d_cen.alloc(3 * (size_t)(nd + mt)));
  BIE_TRY(d_vals.alloc((size_t)mt * 3 * kTile));
  BIE_TRY(d_region.alloc((size_t)chunk * nd));
  DevBuf<unsigned> d_list, d_count;
  BIE_TRY(d_list.alloc((size_t)chunk * nd));
  BIE_TRY(d_count.alloc(1));
  BIE_TRY(d_tm.alloc((size_t)mt * nd));
  BIE_CUDA_TRY(cudaMemcpyAsync(d_cen.ptr, g->centre_d.ptr, 3 * nd * sizeof(double), cudaMemcpyDeviceToDevice, s));
  std::vector<TileMask> tm((size_t)mt * nd);
  std::vector<std::pair<long long, int>> near;  // (point, drop) pairs in Omega_2
  long long all_sources = 0;
  for (int j = 0; j < nd; ++j) all_sources += ngrid(g->p[j]);
  const long long cap_global = std::max<long long>(2048, std::min<long long>(65536, all_sources / (8LL * ctx->sms)));
  auto popc = [](const unsigned* m) {
    int c = 0;
    for (int q = 0; q < 4; ++q) c += __builtin_popcount(m[q]);
    return c;
  };
  for (long long t0 = 0; t0 < npt; t0 += chunk) {
    const long long n = std::min(chunk, npt - t0);
    const int ntile = (int)((n + kTile - 1) / kTile);
    std::vector<int> h_n(ntile, kTile);
    h_n[ntile - 1] = (int)(n - (long long)(ntile - 1) * kTile);
    std::vector<PairItem> items;
    std::vector<int> blk_item, tile_blk(ntile + 1, 0);
    {
      Phase ph(ctx, "offsurface_classify", s);
      BIE_TRY(d_n.upload(h_n));
      BIE_TRY(launch_point_records(pts, npt, t0, n, ntile, nd, d_rec.ptr, d_cen.ptr, s));
      BIE_TRY(launch_classify_points(pts, npt, t0, n, nd, g->centre_d.ptr, d_bnd.ptr, d_h.ptr, ctx->cfg.a_tilde,
                                     g->rec_up.ptr, d_uoff.ptr, d_un.ptr, d_region.ptr, d_list.ptr, d_count.ptr,
                                     ctx->sms, s));
      BIE_TRY(launch_tile_masks(d_region.ptr, nd, d_t0.ptr, d_n.ptr, ntile, d_tm.ptr, s));
      BIE_CUDA_TRY(cudaMemcpyAsync(tm.data(), d_tm.ptr, (size_t)ntile * nd * sizeof(TileMask), cudaMemcpyDeviceToHost,
                                   s));
      BIE_CUDA_TRY(cudaStreamSynchronize(s));
      for (int ti = 0; ti < ntile; ++ti) {
        std::vector<PairItem> mine;
        long long total = 0;
        for (int j = 0; j < nd; ++j) {
          const TileMask& m = tm[(size_t)ti * nd + j];
          if (m.inside) {
            set_error("a point of the tile starting at point " + std::to_string(t0 + (long long)ti * kTile) +
                      " lies inside drop " + std::to_string(j));
            return BIE_EOVERLAP;
          }
          for (int gk = 0; gk < 2; ++gk) {
            if (!popc(m.m[gk])) continue;
            PairItem it{};
            it.tile = ti;
            it.src_drop = j;
            it.grid = gk;
            it.s0 = gk ? g->up_off[j] : g->tgt_off[j];
            it.s1 = it.s0 + (gk ? g->up_n[j] : (long long)ngrid(g->p[j]));
            for (int q = 0; q < 4; ++q) it.mask[q] = m.m[gk][q];
            mine.push_back(it);
            total += it.s1 - it.s0;
          }
          if (m.m[2][0] | m.m[2][1] | m.m[2][2] | m.m[2][3])
            for (int k = 0; k < h_n[ti]; ++k)
              if ((m.m[2][k >> 5] >> (k & 31)) & 1u) near.emplace_back(t0 + (long long)ti * kTile + k, j);
        }
        const long long cap = std::max(cap_global, (total + 15) / 16);  // at most 16 blocks per tile
        tile_blk[ti] = (int)blk_item.size();
        long long used = cap;
        for (auto it : mine) {
          long long a = it.s0;
          while (a < it.s1) {
            if (used >= cap) {
              blk_item.push_back((int)items.size());
              used = 0;
            }
            const long long take = std::min(it.s1 - a, cap - used);
            PairItem piece = it;
            piece.s0 = a;
            piece.s1 = a + take;
            items.push_back(piece);
            used += take;
            a += take;
          }
        }
      }
    }
    const int nblk = (int)blk_item.size();
    tile_blk[ntile] = nblk;
    if (nblk == 0) continue;
    blk_item.push_back((int)items.size());
    BIE_TRY(d_items.upload(items));
    BIE_TRY(d_blk_item.upload(blk_item));
    BIE_TRY(d_tile_blk.upload(tile_blk));
    BIE_TRY(d_part.alloc((size_t)nblk * 3 * kTile));
    for (int k : kinds) {
      const double* wts = weights(k);
      if (prec == BIE_MIXED) {
        Phase ph(ctx, "offsurface_f32", s);
        BIE_TRY(launch_interdrop<float>(k, g->tpt32, nblk, d_items.ptr, d_blk_item.ptr, d_t0.ptr, d_n.ptr, d_drop.ptr,
                                        d_loc.ptr, d_toff.ptr, d_ngd.ptr, d_rec.ptr, d_cen.ptr, g->sX32.ptr,
                                        g->sN32.ptr, q32[k][0].ptr, g->ntarget, g->uX32.ptr, g->uN32.ptr,
                                        q32[k][1].ptr, g->nup_total, wts, d_part.ptr, s));
      } else if (prec == BIE_DF) {
        Phase ph(ctx, "offsurface_df", s);
        BIE_TRY(launch_interdrop_df(k, nblk, d_items.ptr, d_blk_item.ptr, d_t0.ptr, d_n.ptr, d_drop.ptr, d_loc.ptr,
                                    d_toff.ptr, d_ngd.ptr, d_rec.ptr, d_cen.ptr, g->sX64.ptr, g->sN64.ptr,
                                    q64[k][0].ptr, g->ntarget, g->uX64.ptr, g->uN64.ptr, q64[k][1].ptr, g->nup_total,
                                    wts, d_part.ptr, s));
      } else {
        Phase ph(ctx, "offsurface_f64", s);
        BIE_TRY(launch_interdrop<double>(k, g->tpt64, nblk, d_items.ptr, d_blk_item.ptr, d_t0.ptr, d_n.ptr,
                                         d_drop.ptr, d_loc.ptr, d_toff.ptr, d_ngd.ptr, d_rec.ptr, d_cen.ptr,
                                         g->sX64.ptr, g->sN64.ptr, q64[k][0].ptr, g->ntarget, g->uX64.ptr, g->uN64.ptr,
                                         q64[k][1].ptr, g->nup_total, wts, d_part.ptr, s));
      }
      Phase ph(ctx, "offsurface_reduce", s);
      BIE_CUDA_TRY(cudaMemsetAsync(d_vals.ptr, 0, (size_t)ntile * 3 * kTile * sizeof(double), s));
      BIE_TRY(launch_reduce_tiles(d_part.ptr, d_tile_blk.ptr, d_t0.ptr, d_n.ptr, d_drop.ptr, d_loc.ptr, d_voff.ptr,
                                  d_ngd.ptr, ntile, d_vals.ptr, s));
      BIE_TRY(launch_gather_points(d_vals.ptr, t0, n, npt, out[k], s));
    }
    BIE_CUDA_TRY(cudaStreamSynchronize(s));  // the chunk's host tables are reused
  }
  if (near.empty()) return BIE_OK;
  // Omega_2: interpolation along the normal line through the closest point (Sec. 2.3); the closest
  // points and check points serve both layers
  Phase ph(ctx, "offsurface_near", s);
  const int npair = (int)near.size(), L = ctx->cfg.n_interp;
  std::sort(near.begin(), near.end());
  std::vector<NearPair> pairs(npair);
  std::vector<int> tbeg;
  for (int i = 0; i < npair; ++i) {
    pairs[i].target = near[i].first;
    pairs[i].src_drop = near[i].second;
    if (i == 0 || near[i].first != near[i - 1].first) tbeg.push_back(i);
  }
  const int ntgt = (int)tbeg.size();
  tbeg.push_back(npair);
  DevBuf<NearPair> d_pairs;
  DevBuf<int> d_seed, d_tbeg, d_grid, d_tdrop, d_ngd1;
  DevBuf<double> d_npts, d_cv, c64s, c64u;
  DevBuf<long long> d_tloc, d_voff1;
  BIE_TRY(d_pairs.upload(pairs));
  BIE_TRY(d_seed.alloc(npair));
  {
    Phase phs(ctx, "near_seed", s);
    BIE_TRY(launch_near_seed_points(d_pairs.ptr, npair, pts, npt, g->rec_std.ptr, g->toff.ptr, g->ngd.ptr, d_seed.ptr,
                                    s));
  }
  std::vector<int> hseed(npair);
  std::vector<double> hp(3 * (size_t)npt);
  BIE_CUDA_TRY(cudaMemcpyAsync(hseed.data(), d_seed.ptr, npair * sizeof(int), cudaMemcpyDeviceToHost, s));
  BIE_CUDA_TRY(cudaMemcpyAsync(hp.data(), pts, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<double> x0(3 * (size_t)npair);
  for (int i = 0; i < npair; ++i)
    for (int c = 0; c < 3; ++c) x0[3 * i + c] = hp[c * npt + pairs[i].target];
  BIE_TRY(near_points(ctx, g, pairs, x0, hseed, d_npts, d_grid, s));
  BIE_TRY(d_pairs.upload(pairs));
  BIE_TRY(d_tbeg.upload(tbeg));
  BIE_TRY(near_tables(g));
  BIE_TRY(d_cv.alloc(3 * (size_t)npair * L));
  // results go to out[c][t]: one pseudo-drop holding every point, stride npt
  std::vector<long long> tl(npt);
  for (long long t = 0; t < npt; ++t) tl[t] = t;
  BIE_TRY(d_tloc.upload(tl));
  BIE_TRY(d_tdrop.alloc(npt));
  BIE_CUDA_TRY(cudaMemsetAsync(d_tdrop.ptr, 0, npt * sizeof(int), s));
  const std::vector<long long> vo{0};
  const std::vector<int> ng1{(int)npt};
  BIE_TRY(d_voff1.upload(vo));
  BIE_TRY(d_ngd1.upload(ng1));
  for (int k : kinds) {
    const double* wts = weights(k);
    // the on-surface values of the source drops in this precision, as SH expansions
    if (prec == BIE_MIXED)
      BIE_TRY(self_apply<float>(g, k, raw, dens[k], s));
    else if (prec == BIE_DF)
      BIE_TRY(self_apply<dff>(g, k, raw, dens[k], s));
    else
      BIE_TRY(self_apply<double>(g, k, raw, dens[k], s));
    BIE_TRY(near_snapshot(g, s));
    // the check-point values in FP64 (the interpolation amplifies their errors)
    const double *qs = q64[k][0].ptr, *qu = q64[k][1].ptr;
    if (prec == BIE_MIXED) {
      BIE_TRY(c64s.alloc(3 * g->ntarget));
      BIE_TRY(c64u.alloc(3 * g->nup_total));
      BIE_TRY(source_densities<double>(g, dens[k], c64s.ptr, c64u.ptr, s));
      qs = c64s.ptr;
      qu = c64u.ptr;
    }
    Phase phc(ctx, "near_checks", s);
    BIE_TRY(launch_near_checks<double>(k, d_pairs.ptr, npair, L, d_npts.ptr, d_grid.ptr, g->centre_d.ptr,
                                       g->toff.ptr, g->ngd.ptr, g->up_off_d.ptr, g->up_n_d.ptr, g->sX64.ptr,
                                       g->sN64.ptr, qs, g->ntarget, g->uX64.ptr, g->uN64.ptr, qu, g->nup_total, wts,
                                       d_cv.ptr, s));
    BIE_TRY(launch_near_interp(d_pairs.ptr, d_tbeg.ptr, ntgt, L, k, g->selfcoef.ptr, dens[k], g->coef_off_d.ptr,
                               g->pdeg_d.ptr, g->hdrop_d.ptr, wts, d_cv.ptr, d_tdrop.ptr, d_tloc.ptr, d_voff1.ptr,
                               d_ngd1.ptr, out[k], s));
  }
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  return BIE_OK;
}

}  // namespace bie

// ---------------------------------------------------------------------------------------------
// GMRES helpers (device vectors, host Hessenberg)
// ---------------------------------------------------------------------------------------------
namespace bie {
namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 120;

// partial[i][b] = sum over block b's slice of V_i . w   (i < k)
__global__ void k_multidot(const double* __restrict__ V, long long ldv, const double* __restrict__ w, long long n,
                           int k, double* __restrict__ partial) {
  __shared__ double sh[kRedThreads / 32];
  const int i = blockIdx.y;
  const double* v = V + (long long)i * ldv;
  double acc = 0;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x)
    acc += v[x] * w[x];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int q = 0; q < kRedThreads / 32; ++q) t += sh[q];
    partial[(long long)i * gridDim.x + blockIdx.x] = t;
  }
}

// out[i] = sum_b partial[i][b]: one block per entry, fixed summation order
__global__ void k_sum_partials(const double* __restrict__ partial, int nb, int k, double* __restrict__ out) {
  __shared__ double sh[128];
  const int i = blockIdx.x;
  double t = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) t += partial[(long long)i * nb + b];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[i] = sh[0];
}

// y = a*y
__global__ void k_scale(double a, double* __restrict__ y, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] *= a;
}

// y = a*x + b*y
__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}

// y = (lam+1) u - d   (system operator of Eq. main_eq from the double-layer apply d)
__global__ void k_sysop(const double* __restrict__ lam, const double* __restrict__ u, const double* __restrict__ d,
                        double* __restrict__ y, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (lam[i] + 1.0) * u[i] - d[i];
}

// x += V^T y (y on the device, k entries)
__global__ void k_add_comb(double* __restrict__ x, const double* __restrict__ V, long long ldv,
                           const double* __restrict__ y, int k, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = x[i];
  for (int q = 0; q < k; ++q) t += y[q] * V[(long long)q * ldv + i];
  x[i] = t;
}

// ---- fused Krylov kernels: each block owns one contiguous slice of the vectors; dot products are
// reduced per block, then the last block to finish (threadfence + counter) adds the per-block sums
// in block order, so every result is deterministic.
constexpr int kKryThreads = 256;
constexpr int kKryGroup = 4;  // vectors reduced together

__device__ inline void kry_slice(long long n, long long* x0, long long* x1) {
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  *x0 = (long long)blockIdx.x * chunk;
  *x1 = min(n, *x0 + chunk);
}

// partial[i][block] = V_i . w over the block's slice for i < nv (V_nv = w itself when with_norm)
__device__ void kry_block_dots(const double* __restrict__ V, long long ldv, const double* __restrict__ w, int nv,
                               bool with_norm, long long x0, long long x1, double* __restrict__ partial) {
  __shared__ double sh[kKryThreads / 32][kKryGroup];
  const int nt = nv + (with_norm ? 1 : 0);
  for (int i0 = 0; i0 < nt; i0 += kKryGroup) {
    double a[kKryGroup];
#pragma unroll
    for (int g = 0; g < kKryGroup; ++g) a[g] = 0;
    for (long long x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
      const double wx = w[x];
#pragma unroll
      for (int g = 0; g < kKryGroup; ++g) {
        const int i = i0 + g;
        if (i < nv) a[g] += V[(long long)i * ldv + x] * wx;
        else if (i == nv && with_norm) a[g] += wx * wx;
      }
    }
#pragma unroll
    for (int g = 0; g < kKryGroup; ++g)
      for (int o = 16; o > 0; o >>= 1) a[g] += __shfl_down_sync(0xffffffffu, a[g], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
      for (int g = 0; g < kKryGroup; ++g) sh[threadIdx.x >> 5][g] = a[g];
    __syncthreads();
    if (threadIdx.x < kKryGroup && i0 + (int)threadIdx.x < nt) {
      double t = 0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q][threadIdx.x];
      partial[(long long)(i0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// true in the last block to finish; the counter is reset for the next launch
__device__ inline bool kry_last_block(unsigned* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(counter, 1u);
    last = t == gridDim.x - 1;
    if (last) *counter = 0;
  }
  __syncthreads();
  return last;
}

// out[i] = sum over blocks of partial[i][b], b in order (i < nt), by the last block
__device__ inline void kry_finish(const double* partial, int nt, double* out) {
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    double t = 0;
    for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(partial + (long long)i * gridDim.x + b);
    out[i] = t;
  }
}

// w = (lambda + 1) u - d (system operator of Eq. main_eq), then h = V_i . w for i <= k
__global__ void __launch_bounds__(kKryThreads) k_kry_sysop_dots(const double* __restrict__ lam,
                                                                const double* __restrict__ u,
                                                                const double* __restrict__ d, double* __restrict__ w,
                                                                const double* __restrict__ V, long long n, int k,
                                                                double* __restrict__ partial, unsigned* counter,
                                                                double* __restrict__ h) {
  long long x0, x1;
  kry_slice(n, &x0, &x1);
  for (long long x = x0 + threadIdx.x; x < x1; x += blockDim.x) w[x] = (lam[x] + 1.0) * u[x] - d[x];
  __syncthreads();
  kry_block_dots(V, n, w, k + 1, false, x0, x1, partial);
  if (kry_last_block(counter)) kry_finish(partial, k + 1, h);
}

// w -= V h_prev (i <= k), then h = V_i . w for i <= k and h[k+1] = w . w
__global__ void __launch_bounds__(kKryThreads) k_kry_sub_dots(double* __restrict__ w, const double* __restrict__ V,
                                                              long long n, int k, const double* __restrict__ hprev,
                                                              double* __restrict__ partial, unsigned* counter,
                                                              double* __restrict__ h) {
  long long x0, x1;
  kry_slice(n, &x0, &x1);
  for (long long x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
    double t = w[x];
    for (int i = 0; i <= k; ++i) t -= hprev[i] * V[(long long)i * n + x];
    w[x] = t;
  }
  __syncthreads();
  kry_block_dots(V, n, w, k + 1, true, x0, x1, partial);
  if (kry_last_block(counter)) kry_finish(partial, k + 2, h);
}

// w -= V h2 (i <= k); |w| by a direct sum; then, in the last block, the end of Arnoldi step k: the
// Hessenberg column h1 + h2 with subdiagonal |w|, the previous Givens rotations, the new one, the
// least-squares right-hand side gv, the residual estimate res[k] = |gv[k+1]| and scale = 1/|w|
// (applied to w at the start of the next step).
__global__ void __launch_bounds__(kKryThreads) k_kry_sub_tail(double* __restrict__ w, const double* __restrict__ V,
                                                              long long n, int k, int m,
                                                              const double* __restrict__ h1,
                                                              const double* __restrict__ h2,
                                                              double* __restrict__ partial, unsigned* counter,
                                                              double* __restrict__ H, double* __restrict__ cs,
                                                              double* __restrict__ sn, double* __restrict__ gv,
                                                              double* __restrict__ scale, double* __restrict__ res) {
  long long x0, x1;
  kry_slice(n, &x0, &x1);
  for (long long x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
    double t = w[x];
    for (int i = 0; i <= k; ++i) t -= h2[i] * V[(long long)i * n + x];
    w[x] = t;
  }
  __syncthreads();
  kry_block_dots(V, n, w, 0, true, x0, x1, partial);
  if (!kry_last_block(counter)) return;
  if (threadIdx.x != 0) return;
  double wn2 = 0;
  for (int b = 0; b < (int)gridDim.x; ++b) wn2 += __ldcg(partial + b);
  const double hn = sqrt(wn2);
  for (int i = 0; i <= k; ++i) H[(long long)i * m + k] = h1[i] + h2[i];
  for (int i = 0; i < k; ++i) {
    const double a = H[(long long)i * m + k], b = H[(long long)(i + 1) * m + k];
    H[(long long)i * m + k] = cs[i] * a + sn[i] * b;
    H[(long long)(i + 1) * m + k] = -sn[i] * a + cs[i] * b;
  }
  const double a = H[(long long)k * m + k];
  const double den = hypot(a, hn);
  cs[k] = den > 0 ? a / den : 1.0;
  sn[k] = den > 0 ? hn / den : 0.0;
  H[(long long)k * m + k] = den;
  gv[k + 1] = -sn[k] * gv[k];
  gv[k] = cs[k] * gv[k];
  scale[0] = hn > 0 ? 1.0 / hn : 0.0;
  res[k] = fabs(gv[k + 1]);
}

inline int kry_blocks(long long n) { return (int)std::max(1LL, std::min<long long>(120, (n + 255) / 256)); }

// y = s * y with the scale read from the device
__global__ void k_scale_dev(double* __restrict__ y, const double* __restrict__ scale, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] *= scale[0];
}

// start of a cycle: gv = (beta, 0, ..., 0), V_0 = r / beta
__global__ void k_cycle_start(const double* __restrict__ r, double beta, double* __restrict__ v0, long long n,
                              double* __restrict__ gv, int m) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v0[i] = r[i] / beta;
  if (i <= m) gv[i] = i == 0 ? beta : 0.0;
}

// back substitution y = H^-1 gv on the leading k x k triangle (one thread)
__global__ void k_backsub(const double* __restrict__ H, const double* __restrict__ gv, int k, int m,
                          double* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double t = gv[i];
    for (int q = i + 1; q < k; ++q) t -= H[(long long)i * m + q] * y[q];
    y[i] = t / H[(long long)i * m + i];
  }
}

inline unsigned nblk(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

struct Krylov {
  long long n = 0;
  int m = 0;
  DevBuf<double> V, w, tmp, partial, hdev, r, dx, t;
  DevBuf<double> Hd, csd, snd, gvd, scale, resd, yd;  // Hessenberg, rotations, rhs, residual estimates
  DevBuf<unsigned> counter;                              // last-block counter of the fused kernels
  double* hpin = nullptr;  // pinned host copy of the residual estimates
  int hpin_n = 0;
  std::vector<cudaEvent_t> ev;  // end of each Arnoldi step
  struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
    const void* sig[3] = {nullptr, nullptr, nullptr};  // V, tmp, hpin the graph was captured with
  };
  std::map<long long, StepGraph> steps;  // captured Arnoldi steps by (precision, restart, k)
  bool steps_failed = false;             // a capture failed: step eagerly from then on
  ~Krylov() {
    if (hpin) cudaFreeHost(hpin);
    for (auto e : ev) cudaEventDestroy(e);
    for (auto& kv : steps)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  }
};

// out[i] = V_i . w for i < k; with with_norm, out[k] = w . w as well (one synchronisation)
static int dots(Krylov& K, const double* V, int k, const double* w, std::vector<double>& out, cudaStream_t s,
                bool with_norm = false) {
  dim3 grid(kRedBlocks, k);
  k_multidot<<<grid, kRedThreads, 0, s>>>(V, K.n, w, K.n, k, K.partial.ptr);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  if (with_norm) {
    k_multidot<<<dim3(kRedBlocks, 1), kRedThreads, 0, s>>>(w, K.n, w, K.n, 1, K.partial.ptr + (long long)k * kRedBlocks);
    count_launch();
    BIE_CUDA_TRY(cudaGetLastError());
    ++k;
  }
  k_sum_partials<<<k, 128, 0, s>>>(K.partial.ptr, kRedBlocks, k, K.hdev.ptr);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  out.resize(k);
  BIE_CUDA_TRY(cudaMemcpyAsync(out.data(), K.hdev.ptr, k * sizeof(double), cudaMemcpyDeviceToHost, s));
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  return BIE_OK;
}

// |a| and |b| with one synchronisation
static int norm2_pair(Krylov& K, const double* a, const double* b, double* na, double* nb, cudaStream_t s) {
  k_multidot<<<dim3(kRedBlocks, 1), kRedThreads, 0, s>>>(a, K.n, a, K.n, 1, K.partial.ptr);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  k_multidot<<<dim3(kRedBlocks, 1), kRedThreads, 0, s>>>(b, K.n, b, K.n, 1, K.partial.ptr + kRedBlocks);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  k_sum_partials<<<2, 128, 0, s>>>(K.partial.ptr, kRedBlocks, 2, K.hdev.ptr);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  BIE_CUDA_TRY(cudaMemcpyAsync(K.hpin, K.hdev.ptr, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  *na = std::sqrt(std::max(0.0, K.hpin[0]));
  *nb = std::sqrt(std::max(0.0, K.hpin[1]));
  return BIE_OK;
}

static int norm2(Krylov& K, const double* x, double* out, cudaStream_t s) {
  std::vector<double> h;
  BIE_TRY(dots(K, x, 1, x, h, s));
  *out = std::sqrt(std::max(0.0, h[0]));
  return BIE_OK;
}

// system matvec y = (lambda+1) u - D[u] at precision prec
static int sys_matvec(bie_ctx* ctx, const bie_geom* g, const double* u, double* y, double* tmp, int prec,
                      bie_solve_info* info, cudaStream_t s) {
  BIE_TRY(layer_apply(ctx, g, 1, u, tmp, prec, s));
  if (prec == BIE_MIXED)
    info->applies_mixed++;
  else
    info->applies_fp64++;
  Phase ph(ctx, "gmres_vec", s);
  k_sysop<<<nblk(g->ncoef_total), 256, 0, s>>>(g->lamc.ptr, u, tmp, y, g->ncoef_total);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

// Arnoldi step k on stream s: normalisation of V_k (deferred from step k - 1), the operator apply
// into the temporary t2 (its kernels launched one by one when eager_apply), the three fused
// Gram-Schmidt kernels and the copy of the residual estimate to the pinned host array.
static int arnoldi_step(bie_ctx* ctx, const bie_geom* g, Krylov& K, int prec, int k, int m, bool eager_apply,
                        cudaStream_t s) {
  const long long n = g->ncoef_total;
  double* V = K.V.ptr;
  double* t2 = K.tmp.ptr + n;
  double* vk = V + (long long)k * n;
  double* vk1 = V + (long long)(k + 1) * n;
  if (k > 0) {
    k_scale_dev<<<nblk(n), 256, 0, s>>>(vk, K.scale.ptr, n);
    count_launch();
    BIE_CUDA_TRY(cudaGetLastError());
  }
  if (eager_apply)
    BIE_TRY(layer_apply_eager(ctx, g, 1, vk, t2, prec, s));
  else
    BIE_TRY(layer_apply(ctx, g, 1, vk, t2, prec, s));
  double* h1 = K.hdev.ptr;
  double* h2d = K.hdev.ptr + (m + 2);
  const int nbk = kry_blocks(n);
  k_kry_sysop_dots<<<nbk, kKryThreads, 0, s>>>(g->lamc.ptr, vk, t2, vk1, V, n, k, K.partial.ptr, K.counter.ptr, h1);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  k_kry_sub_dots<<<nbk, kKryThreads, 0, s>>>(vk1, V, n, k, h1, K.partial.ptr, K.counter.ptr, h2d);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  k_kry_sub_tail<<<nbk, kKryThreads, 0, s>>>(vk1, V, n, k, m, h1, h2d, K.partial.ptr, K.counter.ptr, K.Hd.ptr,
                                             K.csd.ptr, K.snd.ptr, K.gvd.ptr, K.scale.ptr, K.resd.ptr);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  BIE_CUDA_TRY(cudaMemcpyAsync(K.hpin + k, K.resd.ptr + k, sizeof(double), cudaMemcpyDeviceToHost, s));
  return BIE_OK;
}

// Arnoldi step k as a CUDA graph: captured on the geometry's capture stream at its first use (once
// the operator apply of this precision has run eagerly, so nothing allocates inside the capture) and
// replayed on s after that.  Falls back to launching the step's kernels one by one.
static int arnoldi_step_graph(bie_ctx* ctx, const bie_geom* gc, Krylov& K, int prec, int k, int m,
                              cudaStream_t s) {
  bie_geom* g = const_cast<bie_geom*>(gc);
  const int key_apply = (prec & 0x3ff) * 2 + 1;
  auto ap = g->graphs.find(key_apply);
  const bool warm = ap != g->graphs.end() && ap->second.warm;
  if (!ctx->cfg.use_graphs || ctx->prof.on || !warm || K.steps_failed)
    return arnoldi_step(ctx, gc, K, prec, k, m, false, s);
  const long long key = ((long long)prec * 128 + m) * 128 + k;
  auto& sg = K.steps[key];
  const void* sig[3] = {K.V.ptr, K.tmp.ptr, K.hpin};
  if (sg.exec && (sg.sig[0] != sig[0] || sg.sig[1] != sig[1] || sg.sig[2] != sig[2])) {
    cudaGraphExecDestroy(sg.exec);  // workspace moved since the capture
    sg.exec = nullptr;
  }
  if (!sg.exec) {
    if (!g->cap_stream) BIE_CUDA_TRY(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    const long long l0 = bie_launch_count();
    BIE_CUDA_TRY(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeRelaxed));
    const int st = arnoldi_step(ctx, gc, K, prec, k, m, true, g->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(g->cap_stream, &graph);
    cudaError_t ie = cudaErrorUnknown;
    if (st == BIE_OK && ce == cudaSuccess) ie = cudaGraphInstantiate(&sg.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (st != BIE_OK || ce != cudaSuccess || ie != cudaSuccess) {
      sg.exec = nullptr;
      K.steps_failed = true;
      cudaGetLastError();  // clear the capture's error state
      return arnoldi_step(ctx, gc, K, prec, k, m, false, s);
    }
    sg.launches = bie_launch_count() - l0;
    count_launch(-(int)sg.launches);  // captured, not run
    for (int i = 0; i < 3; ++i) sg.sig[i] = sig[i];
  }
  BIE_CUDA_TRY(cudaGraphLaunch(sg.exec, s));
  count_launch((int)sg.launches);
  return BIE_OK;
}

// Restarted GMRES (Sec. 6) with classical Gram-Schmidt and one re-orthogonalisation, FP64 Krylov
// basis; the operator is applied at precision prec.  x holds the initial guess (zero if x_is_zero).
// Each Arnoldi step runs as the operator apply and three fused kernels that end on the device
// (k_kry_sub_tail); the host reads the residual estimate of step k - 1 after it has queued step k,
// so the device never waits for the host between steps.  A cycle that converges at step k - 1 has
// computed one more step than it uses.
//
// bnorm_in >= 0 is |b| when the caller knows it.  With trust_estimate (the inner solve of the mixed
// refinement, whose true residual the caller recomputes), a cycle that reaches tol by the Givens
// residual estimate returns without recomputing b - A x.
static int gmres(bie_ctx* ctx, const bie_geom* g, int prec, const double* b, double* x, bool x_is_zero, double tol,
                 int restart, int max_iter, Krylov& K, bie_solve_info* info, double* relres, cudaStream_t s,
                 double bnorm_in = -1.0, bool trust_estimate = false) {
  const long long n = g->ncoef_total;
  const int m = restart;
  double* r = K.tmp.ptr;            // residual
  double* t2 = K.tmp.ptr + n;       // apply temporary
  double bnorm = bnorm_in;
  if (bnorm < 0) BIE_TRY(norm2(K, b, &bnorm, s));
  if (bnorm == 0.0) {
    BIE_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    *relres = 0;
    return BIE_OK;
  }
  if (!x_is_zero) {  // a zero initial guess needs no operator apply for its residual
    double xn;
    BIE_TRY(norm2(K, x, &xn, s));
    x_is_zero = xn == 0.0;
  }
  int it = 0;
  while (true) {
    // r = b - A x
    if (x_is_zero) {
      BIE_CUDA_TRY(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      BIE_TRY(sys_matvec(ctx, g, x, r, t2, prec, info, s));
      k_axpby<<<nblk(n), 256, 0, s>>>(1.0, b, -1.0, r, n);
      count_launch();
      BIE_CUDA_TRY(cudaGetLastError());
    }
    double beta;
    if (x_is_zero)
      beta = bnorm;
    else
      BIE_TRY(norm2(K, r, &beta, s));
    *relres = beta / bnorm;
    if (beta / bnorm <= tol || it >= max_iter) return beta / bnorm <= tol ? BIE_OK : BIE_ENOCONV;
    double* V = K.V.ptr;
    k_cycle_start<<<nblk(std::max<long long>(n, m + 1)), 256, 0, s>>>(r, beta, V, n, K.gvd.ptr, m);
    count_launch();
    BIE_CUDA_TRY(cudaGetLastError());
    const int kmax = std::min(m, max_iter - it);
    int k_used = -1;
    double est = beta / bnorm;
    for (int k = 0; k < kmax; ++k) {
      BIE_TRY(arnoldi_step_graph(ctx, g, K, prec, k, m, s));
      if (prec == BIE_MIXED)
        info->applies_mixed++;
      else
        info->applies_fp64++;
      BIE_CUDA_TRY(cudaEventRecord(K.ev[k], s));
      if (k >= 1) {  // step k - 1, read while step k runs
        BIE_CUDA_TRY(cudaEventSynchronize(K.ev[k - 1]));
        const double prev = est;
        est = K.hpin[k - 1] / bnorm;
        if (est <= tol) {
          k_used = k;
          break;
        }
        // when the residual's trend says step k is likely the last one, wait for it before
        // queueing step k + 1 (instead of computing a step that would not be used)
        const double rate = prev > 0 ? est / prev : 1.0;
        if (k + 1 < kmax && est * rate <= 2.0 * tol) {
          BIE_CUDA_TRY(cudaEventSynchronize(K.ev[k]));
          est = K.hpin[k] / bnorm;
          if (est <= tol) {
            k_used = k + 1;
            break;
          }
        }
      }
    }
    if (k_used < 0) {
      BIE_CUDA_TRY(cudaEventSynchronize(K.ev[kmax - 1]));
      est = K.hpin[kmax - 1] / bnorm;
      k_used = kmax;
    }
    it += k_used;
    info->iterations += k_used;
    k_backsub<<<1, 32, 0, s>>>(K.Hd.ptr, K.gvd.ptr, k_used, m, K.yd.ptr);
    count_launch();
    BIE_CUDA_TRY(cudaGetLastError());
    k_add_comb<<<nblk(n), 256, 0, s>>>(x, V, n, K.yd.ptr, k_used, n);
    count_launch();
    BIE_CUDA_TRY(cudaGetLastError());
    x_is_zero = false;
    if (trust_estimate && est <= tol) {
      *relres = est;
      return BIE_OK;
    }
  }
}

}  // namespace bie

namespace bie {
// Velocity of the drop surfaces (Eq. main_eq) for the shapes x and surfactant gamma: geometry,
// interfacial force, far field u_inf = (shear z, 0, 0) (the z coefficients of x, scaled), the
// right-hand side at precision rprec and the solve, into u.  f, uinf and b are n-long temporaries.
static int velocity_solve(bie_ctx* ctx, int ndrop, const int* p, const int* pq, const std::vector<long long>& off,
                          long long n, const double* x, const double* gammacoef, double elasticity, double x_s,
                          const double* lambda, double shear, const bie_solve_opts* opts, int rprec, double* f,
                          double* uinf, double* b, double* u, bie_solve_info* inf, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  bie_geom* g = nullptr;
  BIE_TRY(bie_geometry_setup(ctx, ndrop, p, pq, x, lambda, &g, stream));
  int st = bie_interfacial_force(ctx, g, gammacoef, elasticity, x_s, f, stream);
  if (st == BIE_OK) {
    if (cudaMemsetAsync(uinf, 0, n * sizeof(double), s) != cudaSuccess) st = BIE_ECUDA;
    for (int d = 0; d < ndrop && st == BIE_OK; ++d) {
      const long long nc = ncoef(p[d]);
      if (cudaMemcpyAsync(uinf + off[d], x + off[d] + 2 * nc, nc * sizeof(double), cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
        st = BIE_ECUDA;
    }
    if (st == BIE_OK) {
      k_scale<<<nblk(n), 256, 0, s>>>(shear, uinf, n);
      count_launch();
      if (cudaGetLastError() != cudaSuccess) st = BIE_ECUDA;
    }
  }
  if (st == BIE_OK) st = bie_rhs(ctx, g, uinf, f, b, rprec, stream);
  if (st == BIE_OK && cudaMemsetAsync(u, 0, n * sizeof(double), s) != cudaSuccess) st = BIE_ECUDA;
  if (st == BIE_OK) st = bie_solve(ctx, g, b, u, opts, inf, stream);
  bie_geometry_destroy(g);
  return st;
}
}  // namespace bie

// ---------------------------------------------------------------------------------------------
// surfactant transport (Eq. surfactant0, Sec. 1.2, Sec. 3)
// ---------------------------------------------------------------------------------------------
namespace bie {

// Drops of one degree p on the grid of degree P: device offsets of their vector coefficient sets
// (x, u: [drop][3] blocks, one offset per component) and of their scalar sets (Gamma: [drop]).
struct SurfGroup {
  int p = 0, P = 0;
  Plan* pl = nullptr;
  std::vector<int> drops;
  DevBuf<long long> voff, soff;
};

struct SurfLayout {
  int ndrop = 0;
  std::vector<int> p;
  std::vector<long long> voff, soff;  // per drop: start of its vector / scalar coefficients
  long long nv = 0, ns = 0;           // total lengths
  std::vector<std::unique_ptr<SurfGroup>> groups;
};

// P = 2p + 1 (the nonlinear terms of Sec. 1.3) when upsampled, else P = p.
static int surf_layout(bie_ctx* ctx, int ndrop, const int* p, bool upsampled, SurfLayout& L) {
  L.ndrop = ndrop;
  L.p.assign(p, p + ndrop);
  L.voff.resize(ndrop);
  L.soff.resize(ndrop);
  std::map<int, std::vector<int>> byp;
  for (int d = 0; d < ndrop; ++d) {
    L.voff[d] = L.nv;
    L.soff[d] = L.ns;
    L.nv += 3 * ncoef(p[d]);
    L.ns += ncoef(p[d]);
    byp[p[d]].push_back(d);
  }
  for (auto& kv : byp) {
    std::unique_ptr<SurfGroup> G(new SurfGroup());
    G->p = kv.first;
    G->P = upsampled ? 2 * kv.first + 1 : kv.first;
    BIE_TRY(get_plan(ctx, G->p, G->P, &G->pl));
    G->drops = kv.second;
    std::vector<long long> vo, so;
    for (int d : G->drops) {
      for (int c = 0; c < 3; ++c) vo.push_back(L.voff[d] + c * ncoef(G->p));
      so.push_back(L.soff[d]);
    }
    BIE_TRY(G->voff.upload(vo));
    BIE_TRY(G->soff.upload(so));
    L.groups.push_back(std::move(G));
  }
  return BIE_OK;
}

// Derivative fields of nfield coefficient sets (device offsets off) of the group's degree on its
// grid: kind k (0 f, 1 t, 2 p, 3 tt, 4 tp, 5 pp) is written to out + k * nfield * N.  H holds
// nfield * (p+1) * (P+1) * 2 doubles.
static int surf_synth(const SurfGroup& G, const double* coef, const long long* off, long long nfield,
                      std::initializer_list<int> kinds, double* H, double* out, cudaStream_t s) {
  const Plan* pl = G.pl;
  const double* T[6] = {pl->T0.ptr, pl->T1.ptr, pl->T0.ptr, pl->T2.ptr, pl->T1.ptr, pl->T0.ptr};
  const int dphi[6] = {0, 0, 1, 0, 1, 2};
  const long long N = ngrid(G.P);
  for (int k : kinds) {
    BIE_TRY((launch_leg_synth<double, double>(coef, off, 0, nfield, G.p, T[k], G.P + 1, H, dphi[k], s)));
    BIE_TRY((launch_phi_synth<double, double>(H, nfield, G.p, G.P, pl->cs.ptr, out + (long long)k * nfield * N,
                                              nullptr, N, s)));
  }
  return BIE_OK;
}

static long long synth_work(const SurfGroup& G, long long nfield) {
  return nfield * (G.p + 1) * (long long)(G.P + 1) * 2;
}

// Galerkin projections of f_E and (when fi is non-null) f_I = inv_pe lap Gamma, Sec. 3.
static int surf_rates(const SurfLayout& L, const double* x, const double* u, const double* gam, double inv_pe,
                      double* fe, double* fi, cudaStream_t s) {
  for (auto& Gp : L.groups) {
    const SurfGroup& G = *Gp;
    const long long nd = (long long)G.drops.size(), N = ngrid(G.P);
    const long long nH = synth_work(G, 3 * nd);
    DevBuf<double> tmp;
    BIE_TRY(tmp.alloc(nH + 18 * nd * N + 9 * nd * N + 6 * nd * N + 2 * nd * N));
    double* H = tmp.ptr;
    double* X = H + nH;
    double* U = X + 18 * nd * N;
    double* Gm = U + 9 * nd * N;
    double* out = Gm + 6 * nd * N;
    BIE_TRY(surf_synth(G, x, G.voff.ptr, 3 * nd, {0, 1, 2, 3, 4, 5}, H, X, s));
    BIE_TRY(surf_synth(G, u, G.voff.ptr, 3 * nd, {0, 1, 2}, H, U, s));
    BIE_TRY(surf_synth(G, gam, G.soff.ptr, nd, {0, 1, 2, 3, 4, 5}, H, Gm, s));
    BIE_TRY(launch_surf_rates(X, U, Gm, nd, N, inv_pe, out, fi ? out + nd * N : nullptr, s));
    // H is free again: it serves as the analysis workspace (nd fields need less than 3 nd)
    BIE_TRY(launch_analyze(out, nullptr, N, nd, G.P, G.p, G.pl->cs.ptr, G.pl->A.ptr, H, fe, G.soff.ptr, 0, s));
    if (fi)
      BIE_TRY(launch_analyze(out + nd * N, nullptr, N, nd, G.P, G.p, G.pl->cs.ptr, G.pl->A.ptr, H, fi, G.soff.ptr,
                             0, s));
    BIE_CUDA_TRY(cudaStreamSynchronize(s));  // temporaries are released per group
  }
  return BIE_OK;
}

// Per-drop integrals on the grid of each group (mode 0: volume of x, mode 1: mass of Gamma), host out[d].
static int surf_integrals(const SurfLayout& L, const double* x, const double* gam, int mode, double* out,
                          cudaStream_t s) {
  for (auto& Gp : L.groups) {
    const SurfGroup& G = *Gp;
    const long long nd = (long long)G.drops.size(), N = ngrid(G.P);
    const long long nH = synth_work(G, 3 * nd);
    DevBuf<double> tmp;
    BIE_TRY(tmp.alloc(nH + 9 * nd * N + nd * N + nd));
    double* H = tmp.ptr;
    double* X = H + nH;
    double* Gm = X + 9 * nd * N;
    double* res = Gm + nd * N;
    if (mode == 0)
      BIE_TRY(surf_synth(G, x, G.voff.ptr, 3 * nd, {0, 1, 2}, H, X, s));
    else
      BIE_TRY(surf_synth(G, x, G.voff.ptr, 3 * nd, {1, 2}, H, X, s));
    if (mode == 1) BIE_TRY(surf_synth(G, gam, G.soff.ptr, nd, {0}, H, Gm, s));
    BIE_TRY(launch_drop_integral(X, Gm, nd, G.P, G.pl->wsin.ptr, mode, res, s));
    std::vector<double> h(nd);
    BIE_CUDA_TRY(cudaMemcpyAsync(h.data(), res, nd * sizeof(double), cudaMemcpyDeviceToHost, s));
    BIE_CUDA_TRY(cudaStreamSynchronize(s));
    for (long long i = 0; i < nd; ++i) out[G.drops[i]] = h[i];
  }
  return BIE_OK;
}

// Per-drop max |value| on the grid of each group of ncomp-component coefficient sets (ncomp 3:
// vector layout, 1: scalar layout), host out[d].
static int surf_absmax(const SurfLayout& L, const double* coef, int ncomp, double* out, cudaStream_t s) {
  for (auto& Gp : L.groups) {
    const SurfGroup& G = *Gp;
    const long long nd = (long long)G.drops.size(), N = ngrid(G.P), nf = ncomp * nd;
    const long long nH = synth_work(G, nf);
    DevBuf<double> tmp;
    BIE_TRY(tmp.alloc(nH + nf * N + nd));
    double* H = tmp.ptr;
    double* F = H + nH;
    double* res = F + nf * N;
    BIE_TRY(surf_synth(G, coef, ncomp == 3 ? G.voff.ptr : G.soff.ptr, nf, {0}, H, F, s));
    BIE_TRY(launch_drop_absmax(F, nd, ncomp, N, res, s));
    std::vector<double> h(nd);
    BIE_CUDA_TRY(cudaMemcpyAsync(h.data(), res, nd * sizeof(double), cudaMemcpyDeviceToHost, s));
    BIE_CUDA_TRY(cudaStreamSynchronize(s));
    for (long long i = 0; i < nd; ++i) out[G.drops[i]] = h[i];
  }
  return BIE_OK;
}

// The implicit operator of Sec. 3 (Preconditioning) for the shapes x, left-preconditioned:
// y -> (y - a lap y) / (1 + a n(n+1)/R_d^2), R_d the mean radius of drop d.
struct SurfImplicit {
  const SurfLayout* L = nullptr;
  double a = 0;
  std::vector<std::unique_ptr<DevBuf<double>>> lapc;  // per group [5][nd][N]
  DevBuf<double> inv_diag, c, work;
};

static int surf_implicit_setup(const SurfLayout& L, const double* x, double a, SurfImplicit& I, cudaStream_t s) {
  I.L = &L;
  I.a = a;
  long long wmax = 0;
  for (auto& Gp : L.groups) {
    const SurfGroup& G = *Gp;
    const long long nd = (long long)G.drops.size(), N = ngrid(G.P);
    const long long nH = synth_work(G, 3 * nd);
    DevBuf<double> tmp;
    BIE_TRY(tmp.alloc(nH + 18 * nd * N));
    BIE_TRY(surf_synth(G, x, G.voff.ptr, 3 * nd, {0, 1, 2, 3, 4, 5}, tmp.ptr, tmp.ptr + nH, s));
    std::unique_ptr<DevBuf<double>> lc(new DevBuf<double>());
    BIE_TRY(lc->alloc(5 * nd * N));
    BIE_TRY(launch_lap_coef(tmp.ptr + nH, nd, N, lc->ptr, s));
    BIE_CUDA_TRY(cudaStreamSynchronize(s));
    I.lapc.push_back(std::move(lc));
    wmax = std::max(wmax, synth_work(G, nd) + 7 * nd * N);
  }
  std::vector<double> vol(L.ndrop);
  BIE_TRY(surf_integrals(L, x, nullptr, 0, vol.data(), s));
  std::vector<double> inv(L.ns);
  for (int d = 0; d < L.ndrop; ++d) {
    const double R = std::cbrt(3.0 * vol[d] / (4.0 * kPi));
    for (int n = 0; n <= L.p[d]; ++n)
      for (int i = 0; i < 2 * n + 1; ++i)
        inv[L.soff[d] + (long long)n * n + i] = 1.0 / (1.0 + a * n * (n + 1.0) / (R * R));
  }
  BIE_TRY(I.inv_diag.upload(inv));
  BIE_TRY(I.c.alloc(L.ns));
  BIE_TRY(I.work.alloc(wmax));
  return BIE_OK;
}

static int surf_implicit_apply(SurfImplicit& I, const double* y, double* w, cudaStream_t s) {
  const SurfLayout& L = *I.L;
  for (size_t gi = 0; gi < L.groups.size(); ++gi) {
    const SurfGroup& G = *L.groups[gi];
    const long long nd = (long long)G.drops.size(), N = ngrid(G.P);
    double* H = I.work.ptr;
    double* S = H + synth_work(G, nd);  // [6][nd][N], kinds 1..5 used
    double* grid = S + 6 * nd * N;
    BIE_TRY(surf_synth(G, y, G.soff.ptr, nd, {1, 2, 3, 4, 5}, H, S, s));
    BIE_TRY(launch_lap_apply(I.lapc[gi]->ptr, S, nd, N, grid, s));
    BIE_TRY(launch_analyze(grid, nullptr, N, nd, G.P, G.p, G.pl->cs.ptr, G.pl->A.ptr, H, I.c.ptr, G.soff.ptr, 0, s));
  }
  return launch_implicit_combine(y, I.c.ptr, I.a, I.inv_diag.ptr, L.ns, w, s);
}

// Restarted GMRES (classical Gram-Schmidt with one re-orthogonalisation, Givens rotations on the
// host) for op x = b from x = 0; stops on ||b - op x|| <= tol ||b||.
struct SurfKrylov {
  long long n = 0;
  int m = 0;
  DevBuf<double> V, partial, hdev, ydev;
  int init(long long n_, int m_) {
    n = n_;
    m = m_;
    BIE_TRY(V.alloc((size_t)(m + 1) * n));
    BIE_TRY(partial.alloc((size_t)kRedBlocks * (m + 1)));
    BIE_TRY(hdev.alloc(m + 1));
    BIE_TRY(ydev.alloc(m + 1));
    return BIE_OK;
  }
};

// out[i] = V_i . w for i < k (V_i n apart), on the host
static int surf_dots(SurfKrylov& K, const double* V, int k, const double* w, double* out, cudaStream_t s) {
  k_multidot<<<dim3(kRedBlocks, k), kRedThreads, 0, s>>>(V, K.n, w, K.n, k, K.partial.ptr);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  k_sum_partials<<<k, 128, 0, s>>>(K.partial.ptr, kRedBlocks, k, K.hdev.ptr);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  BIE_CUDA_TRY(cudaMemcpyAsync(out, K.hdev.ptr, k * sizeof(double), cudaMemcpyDeviceToHost, s));
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  return BIE_OK;
}

// x += sum_i c_i V_i (c on the host, k entries)
static int surf_comb(SurfKrylov& K, double* x, const double* V, const double* c, int k, cudaStream_t s) {
  BIE_CUDA_TRY(cudaMemcpyAsync(K.ydev.ptr, c, k * sizeof(double), cudaMemcpyHostToDevice, s));
  k_add_comb<<<nblk(K.n), 256, 0, s>>>(x, V, K.n, K.ydev.ptr, k, K.n);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  BIE_CUDA_TRY(cudaStreamSynchronize(s));  // c may change on return
  return BIE_OK;
}

static int surf_gmres(SurfKrylov& K, const std::function<int(const double*, double*)>& op, const double* b,
                      double* x, double tol, int max_it, int* iters, double* relres, cudaStream_t s) {
  const long long n = K.n;
  const int m = K.m;
  double* V = K.V.ptr;
  BIE_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  double bb;
  BIE_TRY(surf_dots(K, b, 1, b, &bb, s));
  const double bnorm = std::sqrt(bb);
  *iters = 0;
  *relres = 0;
  if (bnorm == 0.0) return BIE_OK;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), h(m + 1), h2(m + 1), y(m);
  auto Hr = [&](int i, int k) -> double& { return H[(size_t)i * m + k]; };
  int it = 0;
  bool xzero = true;
  while (true) {
    double* r = V;
    if (xzero) {
      BIE_CUDA_TRY(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      BIE_TRY(op(x, r));
      k_axpby<<<nblk(n), 256, 0, s>>>(1.0, b, -1.0, r, n);
      count_launch();
      BIE_CUDA_TRY(cudaGetLastError());
    }
    double rr;
    BIE_TRY(surf_dots(K, r, 1, r, &rr, s));
    const double beta = std::sqrt(rr);
    *relres = beta / bnorm;
    *iters = it;
    if (beta / bnorm <= tol) return BIE_OK;
    if (it >= max_it) {
      set_error("surfactant implicit solve: GMRES did not converge");
      return BIE_ENOCONV;
    }
    k_scale<<<nblk(n), 256, 0, s>>>(1.0 / beta, r, n);
    count_launch();
    BIE_CUDA_TRY(cudaGetLastError());
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int used = 0;
    for (int k = 0; k < m; ++k) {
      double* w = V + (long long)(k + 1) * n;
      BIE_TRY(op(V + (long long)k * n, w));
      BIE_TRY(surf_dots(K, V, k + 1, w, h.data(), s));
      for (int i = 0; i <= k; ++i) h2[i] = -h[i];
      BIE_TRY(surf_comb(K, w, V, h2.data(), k + 1, s));
      BIE_TRY(surf_dots(K, V, k + 1, w, h2.data(), s));
      for (int i = 0; i <= k; ++i) {
        h[i] += h2[i];
        h2[i] = -h2[i];
      }
      BIE_TRY(surf_comb(K, w, V, h2.data(), k + 1, s));
      double ww;
      BIE_TRY(surf_dots(K, w, 1, w, &ww, s));
      const double hk1 = std::sqrt(ww);
      if (hk1 > 0.0) {
        k_scale<<<nblk(n), 256, 0, s>>>(1.0 / hk1, w, n);
        count_launch();
        BIE_CUDA_TRY(cudaGetLastError());
      }
      for (int i = 0; i <= k; ++i) Hr(i, k) = h[i];
      Hr(k + 1, k) = hk1;
      for (int i = 0; i < k; ++i) {
        const double t = cs[i] * Hr(i, k) + sn[i] * Hr(i + 1, k);
        Hr(i + 1, k) = -sn[i] * Hr(i, k) + cs[i] * Hr(i + 1, k);
        Hr(i, k) = t;
      }
      const double den = std::hypot(Hr(k, k), Hr(k + 1, k));
      cs[k] = Hr(k, k) / den;
      sn[k] = Hr(k + 1, k) / den;
      Hr(k, k) = den;
      Hr(k + 1, k) = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      ++it;
      used = k + 1;
      if (std::fabs(g[k + 1]) / bnorm <= tol || it >= max_it || hk1 == 0.0) break;
    }
    for (int i = used - 1; i >= 0; --i) {
      double t = g[i];
      for (int j = i + 1; j < used; ++j) t -= Hr(i, j) * y[j];
      y[i] = t / Hr(i, i);
    }
    BIE_TRY(surf_comb(K, x, V, y.data(), used, s));
    xzero = false;
  }
}

// y with (I - a lap_x) y = b per drop (Galerkin), left-preconditioned GMRES.
static int surf_implicit_solve(const SurfLayout& L, const double* x, const double* b, double a, double* y,
                               double tol, int* iters, cudaStream_t s) {
  *iters = 0;
  if (a == 0.0) {
    BIE_CUDA_TRY(cudaMemcpyAsync(y, b, L.ns * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return BIE_OK;
  }
  SurfImplicit I;
  BIE_TRY(surf_implicit_setup(L, x, a, I, s));
  DevBuf<double> bp;
  BIE_TRY(bp.alloc(L.ns));
  BIE_TRY(launch_mul(b, I.inv_diag.ptr, L.ns, bp.ptr, s));
  SurfKrylov K;
  BIE_TRY(K.init(L.ns, 60));
  double rel;
  auto op = [&](const double* in, double* out) { return surf_implicit_apply(I, in, out, s); };
  return surf_gmres(K, op, bp.ptr, y, tol, 600, iters, &rel, s);
}

}  // namespace bie

// ---------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------
using namespace bie;

extern "C" {

void bie_config_default(bie_config* cfg) {
  if (!cfg) return;
  cfg->device = 0;
  cfg->upsample = 4;
  cfg->a_tilde = 5.0;
  cfg->n_interp = 8;
  cfg->self_direct = 0;
  cfg->use_graphs = 1;
  cfg->tensor_rotation = 0;
}

const char* bie_strerror(int st) {
  switch (st) {
    case BIE_OK: return "ok";
    case BIE_EINVAL: return "invalid argument";
    case BIE_ENOMEM: return "out of memory";
    case BIE_ECUDA: return "CUDA error";
    case BIE_ENOCONV: return "iterative solve did not converge";
    case BIE_ETIMEOUT: return "bounded device wait timed out";
    case BIE_EOVERLAP: return "drops overlap";
    case BIE_ENOTSUP: return "not supported";
    default: return "unknown status";
  }
}

const char* bie_last_error(void) { return g_last_error.c_str(); }

int bie_create(bie_ctx** out, const bie_config* cfg) {
  if (!out) return BIE_EINVAL;
  *out = nullptr;
  bie_config c;
  bie_config_default(&c);
  if (cfg) c = *cfg;
  if (c.upsample < 1 || c.a_tilde <= 1.0 || c.n_interp < 1 || c.n_interp > 16) {
    set_error("bad config");
    return BIE_EINVAL;
  }
  int ndev = 0;
  BIE_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (c.device < 0 || c.device >= ndev) {
    set_error("device ordinal out of range");
    return BIE_EINVAL;
  }
  BIE_CUDA_TRY(cudaSetDevice(c.device));
  int sms = 0;
  BIE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
  bie_ctx* ctx = new bie_ctx();
  ctx->cfg = c;
  ctx->sms = sms;
  *out = ctx;
  return BIE_OK;
}

void bie_destroy(bie_ctx* ctx) { delete ctx; }

int bie_sh_analyze(bie_ctx* ctx, int ndrop, const int* p, int ncomp, const double* grid, double* coef,
                   void* stream) {
  if (!ctx || !grid || !coef || ncomp <= 0) return BIE_EINVAL;
  BIE_TRY(check_degrees(ndrop, p));
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  long long go = 0, co = 0;
  for (int d = 0; d < ndrop; ++d) {
    Plan* pl;
    BIE_TRY(get_plan(ctx, p[d], p[d], &pl));
    BIE_TRY(ctx->scratch.alloc((size_t)ncomp * (p[d] + 1) * (p[d] + 1) * 2));
    BIE_TRY(launch_analyze(grid + go, nullptr, ngrid(p[d]), ncomp, p[d], p[d], pl->cs.ptr, pl->A.ptr,
                           ctx->scratch.ptr, coef + co, nullptr, ncoef(p[d]), s));
    go += ncomp * ngrid(p[d]);
    co += ncomp * ncoef(p[d]);
  }
  return BIE_OK;
}

int bie_sh_synthesize(bie_ctx* ctx, int ndrop, const int* p, const int* p_out, int ncomp, const double* coef,
                      double* grid, void* stream) {
  if (!ctx || !grid || !coef || !p_out || ncomp <= 0) return BIE_EINVAL;
  BIE_TRY(check_degrees(ndrop, p));
  for (int d = 0; d < ndrop; ++d)
    if (p_out[d] < p[d] || p_out[d] > 4 * BIE_MAX_P) {
      set_error("p_out must satisfy p <= p_out <= 4*BIE_MAX_P");
      return BIE_EINVAL;
    }
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  long long go = 0, co = 0;
  for (int d = 0; d < ndrop; ++d) {
    Plan* pl;
    BIE_TRY(get_plan(ctx, p[d], p_out[d], &pl));
    BIE_TRY(ctx->scratch.alloc((size_t)ncomp * (p[d] + 1) * (p_out[d] + 1) * 2));
    BIE_TRY((launch_leg_synth<double, double>(coef + co, nullptr, ncoef(p[d]), ncomp, p[d], pl->T0.ptr,
                                              p_out[d] + 1, ctx->scratch.ptr, 0, s)));
    BIE_TRY((launch_phi_synth<double, double>(ctx->scratch.ptr, ncomp, p[d], p_out[d], pl->cs.ptr, grid + go,
                                              nullptr, ngrid(p_out[d]), s)));
    go += ncomp * ngrid(p_out[d]);
    co += ncomp * ncoef(p[d]);
  }
  return BIE_OK;
}

int bie_rotate(bie_ctx* ctx, int ndrop, const int* p, int ncomp, const double* coef, const double* euler,
               double* coef_out, void* stream) {
  if (!ctx || !coef || !coef_out || !euler || ncomp <= 0) return BIE_EINVAL;
  BIE_TRY(check_degrees(ndrop, p));
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  long long co = 0;
  for (int d = 0; d < ndrop; ++d) {
    const int pd = p[d];
    std::vector<double> blk(wigner_block_stride(pd));
    wigner_blocks(pd, euler[3 * d + 1], blk.data());
    std::vector<double> ph((size_t)(pd + 1) * 2);
    for (int m = 0; m <= pd; ++m) {
      ph[2 * m] = std::cos(m * euler[3 * d]);
      ph[2 * m + 1] = std::sin(m * euler[3 * d]);
    }
    std::vector<long long> foff(ncomp);
    for (int c = 0; c < ncomp; ++c) foff[c] = co + c * ncoef(pd);
    DevBuf<double> dblk, dph;
    DevBuf<long long> dfo;
    BIE_TRY(dblk.upload(blk));
    BIE_TRY(dph.upload(ph));
    BIE_TRY(dfo.upload(foff));
    BIE_TRY((launch_rotate<double, double>(coef, dfo.ptr, ncomp, 1, pd, dblk.ptr, (long long)blk.size(), 1, 1,
                                           dph.ptr, coef_out + co, 0, s)));
    BIE_TRY(launch_phase(coef_out + co, ncomp, pd, euler[3 * d + 2], s));
    BIE_CUDA_TRY(cudaStreamSynchronize(s));  // the staged tables are released on return
    co += ncomp * ncoef(pd);
  }
  return BIE_OK;
}

int bie_geometry_setup(bie_ctx* ctx, int ndrop, const int* p, const int* pq, const double* xcoef,
                       const double* lambda, bie_geom** out, void* stream) {
  if (!ctx || !out || !xcoef || !lambda || !pq) return BIE_EINVAL;
  *out = nullptr;
  BIE_TRY(check_degrees(ndrop, p));
  for (int d = 0; d < ndrop; ++d)
    if (pq[d] < p[d] || pq[d] > 2 * p[d] + 1) {
      set_error("pq must satisfy p <= pq <= 2p+1");
      return BIE_EINVAL;
    }
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<bie_geom> g(new bie_geom());
  g->ctx = ctx;
  g->ndrop = ndrop;
  g->p.assign(p, p + ndrop);
  g->pq.assign(pq, pq + ndrop);
  g->lambda.assign(lambda, lambda + ndrop);
  g->coef_off.resize(ndrop);
  g->tgt_off.resize(ndrop);
  long long co = 0, to = 0;
  for (int d = 0; d < ndrop; ++d) {
    g->coef_off[d] = co;
    g->tgt_off[d] = to;
    co += 3 * ncoef(p[d]);
    to += ngrid(p[d]);
  }
  g->ncoef_total = co;
  g->ntarget = to;
  BIE_TRY(g->xcoef.alloc(co));
  BIE_CUDA_TRY(cudaMemcpyAsync(g->xcoef.ptr, xcoef, co * sizeof(double), cudaMemcpyDeviceToDevice, s));
  BIE_TRY(g->rec_std.alloc(7 * to));
  BIE_TRY(g->vals.alloc(3 * to));
  {
    std::vector<double> lc(co);
    for (int d = 0; d < ndrop; ++d)
      std::fill(lc.begin() + g->coef_off[d], lc.begin() + g->coef_off[d] + 3 * ncoef(p[d]), lambda[d]);
    BIE_TRY(g->lamc.upload(lc));
  }
  // group drops of equal (p, pq)
  std::map<std::pair<int, int>, int> gi;
  for (int d = 0; d < ndrop; ++d) {
    auto key = std::make_pair(p[d], pq[d]);
    if (!gi.count(key)) {
      gi[key] = (int)g->groups.size();
      g->groups.emplace_back(new bie_geom::Group());
      g->groups.back()->p = p[d];
      g->groups.back()->pq = pq[d];
    }
    g->groups[gi[key]]->drops.push_back(d);
  }
  long long self_pairs = 0;
  for (auto& G : g->groups) {
    BIE_TRY(setup_group(ctx, g.get(), *G, s));
    self_pairs += (long long)G->drops.size() * ngrid(G->p) * ngrid(G->pq);
  }
  if (ndrop > 1) BIE_TRY(setup_interdrop(ctx, g.get(), s));
  // projected-form groups: both kinds' factors now, then the rotated-grid cache is no longer needed
  for (auto& G : g->groups) {
    if (group_uses_direct(ctx, *G)) continue;
    BIE_TRY(ensure_qk(ctx, *G, 0, s));
    BIE_TRY(ensure_qk(ctx, *G, 1, s));
    BIE_CUDA_TRY(cudaStreamSynchronize(s));
    G->cache64.release();
  }
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  g->info.ndrop = ndrop;
  g->info.ncoef = co;
  g->info.ntarget = to;
  g->info.self_pairs = self_pairs;
  double bytes = 0;
  for (auto& G : g->groups)
    bytes += G->cache64.n * 8.0 + (G->qk64[0].n + G->qk64[1].n) * 8.0 + (G->qk32[0].n + G->qk32[1].n) * 4.0;
  bytes += g->rec_std.n * 8.0 + g->vals.n * 8.0 + g->xcoef.n * 8.0;
  g->info.cache_bytes = bytes;
  *out = g.release();
  return BIE_OK;
}

void bie_geometry_destroy(bie_geom* g) {
  if (!g) return;
  for (auto& kv : g->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  delete g->kry;
  delete g;
}

int bie_geometry_info(const bie_geom* g, bie_geom_info* info) {
  if (!g || !info) return BIE_EINVAL;
  *info = g->info;
  return BIE_OK;
}

int bie_interfacial_force(bie_ctx* ctx, const bie_geom* g, const double* gammacoef, double elasticity, double x_s,
                          double* fcoef, void* stream) {
  if (!ctx || !g || !gammacoef || !fcoef) return BIE_EINVAL;
  if (x_s < 0.0 || x_s >= 1.0) {
    set_error("surface coverage x_s must satisfy 0 <= x_s < 1");
    return BIE_EINVAL;
  }
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  Phase phz(ctx, "force", s);
  long long go = 0;  // offset of drop d's Gamma coefficients (one scalar per drop)
  for (int d = 0; d < g->ndrop; ++d) {
    const int p = g->p[d], P = 2 * p + 1;  // nonlinear terms on the grid of degree 2p+1 (Sec. 1.3)
    Plan* pl;
    BIE_TRY(get_plan(ctx, p, P, &pl));
    const long long N = ngrid(P), nc = ncoef(p);
    DevBuf<double> tmp;
    BIE_TRY(tmp.alloc(3 * (p + 1) * (size_t)(P + 1) * 2 + 18 * N + 3 * N + 3 * N + 3 * (p + 1) * (size_t)(P + 1) * 2));
    double* H = tmp.ptr;
    double* X = H + 3 * (p + 1) * (long long)(P + 1) * 2;  // [6][3][N]
    double* Gm = X + 18 * N;                                // [3][N]
    double* f = Gm + 3 * N;                                 // [3][N]
    double* F = f + 3 * N;
    const double* xc = g->xcoef.ptr + g->coef_off[d];
    const double* T[6] = {pl->T0.ptr, pl->T1.ptr, pl->T0.ptr, pl->T2.ptr, pl->T1.ptr, pl->T0.ptr};
    const int dphi[6] = {0, 0, 1, 0, 1, 2};
    for (int k = 0; k < 6; ++k) {
      BIE_TRY((launch_leg_synth<double, double>(xc, nullptr, nc, 3, p, T[k], P + 1, H, dphi[k], s)));
      BIE_TRY((launch_phi_synth<double, double>(H, 3, p, P, pl->cs.ptr, X + k * 3 * N, nullptr, N, s)));
    }
    for (int k = 0; k < 3; ++k) {
      BIE_TRY((launch_leg_synth<double, double>(gammacoef + go, nullptr, nc, 1, p, T[k], P + 1, H, dphi[k], s)));
      BIE_TRY((launch_phi_synth<double, double>(H, 1, p, P, pl->cs.ptr, Gm + k * N, nullptr, N, s)));
    }
    BIE_TRY(launch_force(X, Gm, N, elasticity, x_s, f, s));
    BIE_TRY(launch_analyze(f, nullptr, N, 3, P, p, pl->cs.ptr, pl->A.ptr, F, fcoef + g->coef_off[d], nullptr, nc, s));
    BIE_CUDA_TRY(cudaStreamSynchronize(s));  // the temporaries are released per drop
    go += nc;
  }
  return BIE_OK;
}

int bie_apply_single(bie_ctx* ctx, const bie_geom* g, const double* fcoef, double* out, int precision,
                     void* stream) {
  if (!ctx) return BIE_EINVAL;
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  return layer_apply(ctx, g, 0, fcoef, out, precision, (cudaStream_t)stream);
}

int bie_apply_double(bie_ctx* ctx, const bie_geom* g, const double* ucoef, double* out, int precision,
                     void* stream) {
  if (!ctx) return BIE_EINVAL;
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  return layer_apply(ctx, g, 1, ucoef, out, precision, (cudaStream_t)stream);
}

int bie_eval_single(bie_ctx* ctx, const bie_geom* g, long long npoint, const double* points, const double* fcoef,
                    double* out, int precision, void* stream) {
  if (!ctx || !g || (npoint > 0 && (!points || !fcoef || !out))) return BIE_EINVAL;
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  const double* dens[2] = {fcoef, nullptr};
  double* outs[2] = {out, nullptr};
  return bie::eval_layers(ctx, const_cast<bie_geom*>(g), npoint, points, dens, outs, precision, (cudaStream_t)stream);
}

int bie_eval_double(bie_ctx* ctx, const bie_geom* g, long long npoint, const double* points, const double* ucoef,
                    double* out, int precision, void* stream) {
  if (!ctx || !g || (npoint > 0 && (!points || !ucoef || !out))) return BIE_EINVAL;
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  const double* dens[2] = {nullptr, ucoef};
  double* outs[2] = {nullptr, out};
  return bie::eval_layers(ctx, const_cast<bie_geom*>(g), npoint, points, dens, outs, precision, (cudaStream_t)stream);
}

int bie_eval_velocity(bie_ctx* ctx, const bie_geom* g, long long npoint, const double* points, const double* fcoef,
                      const double* ucoef, const double* uinf, double* out, int precision, void* stream) {
  if (!ctx || !g || (npoint > 0 && (!points || !fcoef || !ucoef || !out))) return BIE_EINVAL;
  if (precision & BIE_RAW) {
    set_error("bie_eval_velocity: BIE_RAW is not a velocity");
    return BIE_EINVAL;
  }
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  if (npoint == 0) return BIE_OK;
  cudaStream_t s = (cudaStream_t)stream;
  bie::DevBuf<double> S, D;
  BIE_TRY(S.alloc(3 * npoint));
  BIE_TRY(D.alloc(3 * npoint));
  const double* dens[2] = {fcoef, ucoef};
  double* outs[2] = {S.ptr, D.ptr};
  BIE_TRY(bie::eval_layers(ctx, const_cast<bie_geom*>(g), npoint, points, dens, outs, precision, s));
  BIE_TRY(bie::launch_velocity(uinf, S.ptr, D.ptr, 3 * npoint, out, s));
  BIE_CUDA_TRY(cudaStreamSynchronize(s));  // S and D are released on return
  return BIE_OK;
}

int bie_rhs(bie_ctx* ctx, const bie_geom* g, const double* uinf, const double* fcoef, double* rhs, int precision,
            void* stream) {
  if (!ctx || !g || !uinf || !fcoef || !rhs) return BIE_EINVAL;
  if (precision != BIE_FP64 && precision != BIE_DF) {
    set_error("bie_rhs: precision must be BIE_FP64 or BIE_DF");
    return BIE_EINVAL;
  }
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  BIE_TRY(layer_apply(ctx, g, 0, fcoef, rhs, precision, s));
  Phase ph(ctx, "gmres_vec", s);
  k_axpby<<<nblk(g->ncoef_total), 256, 0, s>>>(2.0, uinf, 1.0, rhs, g->ncoef_total);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

void bie_solve_opts_default(bie_solve_opts* o) {
  if (!o) return;
  o->precision = BIE_FP64;
  o->tol = 1e-10;
  o->restart = 30;
  o->max_iter = 300;
  o->inner_tol = 1e-5;
  o->max_refine = 10;
  o->residual_precision = BIE_DF;
}

int bie_solve(bie_ctx* ctx, const bie_geom* g, const double* rhs, double* u, const bie_solve_opts* opts,
              bie_solve_info* info, void* stream) {
  if (!ctx || !g || !rhs || !u || !opts || !info) return BIE_EINVAL;
  if (opts->restart < 1 || opts->restart > 64 || opts->tol <= 0 || opts->max_iter < 1 ||
      (opts->residual_precision != BIE_FP64 && opts->residual_precision != BIE_DF)) {
    set_error("bad solve options");
    return BIE_EINVAL;
  }
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  std::memset(info, 0, sizeof(*info));
  const long long n = g->ncoef_total;
  bie_geom* gm = const_cast<bie_geom*>(g);
  if (!gm->kry || gm->kry->m < opts->restart) {
    delete gm->kry;
    gm->kry = new bie::Krylov();
  }
  bie::Krylov& K = *gm->kry;
  K.n = n;
  K.m = opts->restart;
  BIE_TRY(K.V.alloc((size_t)(opts->restart + 1) * n));
  BIE_TRY(K.tmp.alloc(3 * n));
  BIE_TRY(K.partial.alloc((size_t)kRedBlocks * (opts->restart + 2)));
  BIE_TRY(K.hdev.alloc(2 * (opts->restart + 2)));
  const int mr = opts->restart;
  BIE_TRY(K.Hd.alloc((size_t)(mr + 1) * mr));
  BIE_TRY(K.csd.alloc(mr));
  BIE_TRY(K.snd.alloc(mr));
  BIE_TRY(K.gvd.alloc(mr + 1));
  BIE_TRY(K.scale.alloc(1));
  BIE_TRY(K.resd.alloc(mr));
  BIE_TRY(K.yd.alloc(mr));
  if (!K.counter.ptr) {
    BIE_TRY(K.counter.alloc(1));
    BIE_CUDA_TRY(cudaMemset(K.counter.ptr, 0, sizeof(unsigned)));
  }
  if (K.hpin_n < std::max(mr, 2)) {
    if (K.hpin) cudaFreeHost(K.hpin);
    K.hpin = nullptr;
    BIE_CUDA_TRY(cudaMallocHost(&K.hpin, std::max(mr, 2) * sizeof(double)));
    K.hpin_n = std::max(mr, 2);
  }
  while ((int)K.ev.size() < mr) {
    cudaEvent_t e;
    BIE_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    K.ev.push_back(e);
  }
  double rel = 0;
  int st;
  if ((opts->precision & 0xff) == BIE_FP64) {
    st = gmres(ctx, g, BIE_FP64, rhs, u, false, opts->tol, opts->restart, opts->max_iter, K, info, &rel, s);
    info->residual = rel;
    info->converged = st == BIE_OK;
    return st;
  }
  // mixed: FP64 residual outside, mixed-precision GMRES correction inside
  DevBuf<double>&r = K.r, &dx = K.dx, &t = K.t;
  BIE_TRY(r.alloc(n));
  BIE_TRY(dx.alloc(n));
  BIE_TRY(t.alloc(n));
  double bnorm, unorm;
  BIE_TRY(norm2_pair(K, rhs, u, &bnorm, &unorm, s));
  int left = opts->max_iter;
  bool updated = false;
  for (int outer = 0;; ++outer) {
    if (outer == 0 && unorm == 0.0) {  // r = b for a zero initial guess
      BIE_CUDA_TRY(cudaMemcpyAsync(r.ptr, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else if (!updated) {
      BIE_TRY(sys_matvec(ctx, g, u, r.ptr, t.ptr, opts->residual_precision, info, s));
      k_axpby<<<nblk(n), 256, 0, s>>>(1.0, rhs, -1.0, r.ptr, n);
      count_launch();
      BIE_CUDA_TRY(cudaGetLastError());
    }
    double rn;
    if (outer == 0 && unorm == 0.0)
      rn = bnorm;
    else
      BIE_TRY(norm2(K, r.ptr, &rn, s));
    rel = bnorm > 0 ? rn / bnorm : 0.0;
    info->residual = rel;
    if (rel <= opts->tol) {
      info->converged = 1;
      return BIE_OK;
    }
    if (outer >= opts->max_refine || left <= 0) return BIE_ENOCONV;
    info->refinements++;
    int before = info->iterations;
    double inner_rel;
    BIE_CUDA_TRY(cudaMemsetAsync(dx.ptr, 0, n * sizeof(double), s));
    st = gmres(ctx, g, BIE_MIXED, r.ptr, dx.ptr, true, opts->inner_tol, opts->restart, left, K, info, &inner_rel, s,
               rn, true);
    if (st != BIE_OK && st != BIE_ENOCONV) return st;
    left -= info->iterations - before;
    k_axpby<<<nblk(n), 256, 0, s>>>(1.0, dx.ptr, 1.0, u, n);
    count_launch();
    BIE_CUDA_TRY(cudaGetLastError());
    // Next residual.  Once the correction is small against u, r <- r - A dx with the mixed operator
    // is accurate to ~eps_32 |A| |dx|, far below the tolerance; otherwise recompute b - A u in FP64.
    double dxn;
    BIE_TRY(norm2_pair(K, dx.ptr, u, &dxn, &unorm, s));
    if (dxn <= 1e-4 * unorm) {
      BIE_TRY(sys_matvec(ctx, g, dx.ptr, t.ptr, K.tmp.ptr + 2 * n, BIE_MIXED, info, s));
      k_axpby<<<nblk(n), 256, 0, s>>>(-1.0, t.ptr, 1.0, r.ptr, n);
      count_launch();
      BIE_CUDA_TRY(cudaGetLastError());
      updated = true;
    } else {
      updated = false;
    }
  }
}

int bie_step_midpoint(bie_ctx* ctx, int ndrop, const int* p, const int* pq, double* xcoef, const double* gammacoef,
                      double elasticity, double x_s, const double* lambda, double shear, double dt,
                      const bie_solve_opts* opts, bie_solve_info* info, void* stream) {
  if (!ctx || !p || !pq || !xcoef || !gammacoef || !lambda || !opts) {
    set_error("null argument");
    return BIE_EINVAL;
  }
  BIE_TRY(check_degrees(ndrop, p));
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<long long> off(ndrop);
  long long n = 0;
  for (int d = 0; d < ndrop; ++d) {
    off[d] = n;
    n += 3 * ncoef(p[d]);
  }
  DevBuf<double> xh, f, uinf, b, u;
  BIE_TRY(xh.alloc(n));
  BIE_TRY(f.alloc(n));
  BIE_TRY(uinf.alloc(n));
  BIE_TRY(b.alloc(n));
  BIE_TRY(u.alloc(n));
  // the right-hand side at the solve's FP64-grade precision
  const int rprec = (opts->precision & 0xff) == BIE_FP64 ? BIE_FP64 : opts->residual_precision;
  // u(x): Eq. main_eq for the shapes x with the surfactant held fixed
  auto velocity = [&](const double* x, bie_solve_info* inf) -> int {
    return velocity_solve(ctx, ndrop, p, pq, off, n, x, gammacoef, elasticity, x_s, lambda, shear, opts, rprec, f.ptr,
                          uinf.ptr, b.ptr, u.ptr, inf, stream);
  };
  bie_solve_info tmp[2];
  bie_solve_info* inf = info ? info : tmp;
  BIE_TRY(velocity(xcoef, &inf[0]));
  // x^{1/2} = x + (dt/2) u(x)
  BIE_CUDA_TRY(cudaMemcpyAsync(xh.ptr, xcoef, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  k_axpby<<<nblk(n), 256, 0, s>>>(0.5 * dt, u.ptr, 1.0, xh.ptr, n);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  BIE_TRY(velocity(xh.ptr, &inf[1]));
  // x^{new} = x + dt u(x^{1/2})
  k_axpby<<<nblk(n), 256, 0, s>>>(dt, u.ptr, 1.0, xcoef, n);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  return BIE_OK;
}

int bie_profile(bie_ctx* ctx, int enable) {
  if (!ctx) return BIE_EINVAL;
  ctx->prof.on = enable != 0;
  ctx->prof.used = 0;
  ctx->prof.recs.clear();
  return BIE_OK;
}

int bie_profile_read(bie_ctx* ctx, bie_phase_stat* stats, int cap, int* count) {
  if (!ctx || !count || (cap > 0 && !stats)) return BIE_EINVAL;
  auto& P = ctx->prof;
  std::vector<std::string> names;
  std::vector<double> ms;
  std::vector<long long> n;
  for (auto& r : P.recs) {
    BIE_CUDA_TRY(cudaEventSynchronize(P.pool[r.second + 1]));
    float t = 0;
    BIE_CUDA_TRY(cudaEventElapsedTime(&t, P.pool[r.second], P.pool[r.second + 1]));
    size_t k = std::find(names.begin(), names.end(), r.first) - names.begin();
    if (k == names.size()) {
      names.push_back(r.first);
      ms.push_back(0);
      n.push_back(0);
    }
    ms[k] += t;
    n[k] += 1;
  }
  *count = (int)names.size();
  for (int i = 0; i < (int)names.size() && i < cap; ++i) {
    std::memset(stats[i].name, 0, sizeof(stats[i].name));
    std::strncpy(stats[i].name, names[i].c_str(), sizeof(stats[i].name) - 1);
    stats[i].ms = ms[i];
    stats[i].calls = n[i];
  }
  P.used = 0;
  P.recs.clear();
  return BIE_OK;
}

static int surf_check(bie_ctx* ctx, int ndrop, const int* p) {
  if (!ctx) {
    set_error("null argument");
    return BIE_EINVAL;
  }
  BIE_TRY(check_degrees(ndrop, p));
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  return BIE_OK;
}

int bie_surfactant_rates(bie_ctx* ctx, int ndrop, const int* p, const double* xcoef, const double* ucoef,
                         const double* gammacoef, double inv_pe, double* fe, double* fi, void* stream) {
  if (!xcoef || !ucoef || !gammacoef || !fe || inv_pe < 0.0) {
    set_error("null argument or negative 1/Pe");
    return BIE_EINVAL;
  }
  BIE_TRY(surf_check(ctx, ndrop, p));
  cudaStream_t s = (cudaStream_t)stream;
  Phase ph(ctx, "surfactant_rates", s);
  SurfLayout L;
  BIE_TRY(surf_layout(ctx, ndrop, p, true, L));
  return surf_rates(L, xcoef, ucoef, gammacoef, inv_pe, fe, fi, s);
}

int bie_surfactant_implicit(bie_ctx* ctx, int ndrop, const int* p, const double* xcoef, const double* b, double a,
                            double* y, double tol, int* iterations, void* stream) {
  if (!xcoef || !b || !y || a < 0.0 || !(tol > 0.0)) {
    set_error("null argument, negative a or non-positive tol");
    return BIE_EINVAL;
  }
  BIE_TRY(surf_check(ctx, ndrop, p));
  cudaStream_t s = (cudaStream_t)stream;
  Phase ph(ctx, "surfactant_implicit", s);
  SurfLayout L;
  BIE_TRY(surf_layout(ctx, ndrop, p, true, L));
  int it = 0;
  const int st = surf_implicit_solve(L, xcoef, b, a, y, tol, &it, s);
  if (iterations) *iterations = it;
  return st;
}

int bie_surfactant_mass(bie_ctx* ctx, int ndrop, const int* p, const double* xcoef, const double* gammacoef,
                        double* mass, void* stream) {
  if (!xcoef || !gammacoef || !mass) {
    set_error("null argument");
    return BIE_EINVAL;
  }
  BIE_TRY(surf_check(ctx, ndrop, p));
  SurfLayout L;
  BIE_TRY(surf_layout(ctx, ndrop, p, true, L));
  return surf_integrals(L, xcoef, gammacoef, 1, mass, (cudaStream_t)stream);
}

int bie_step_coupled(bie_ctx* ctx, int ndrop, const int* p, const int* pq, const double* xcoef,
                     const double* gammacoef, double* u0, int u0_valid, double elasticity, double x_s,
                     const double* lambda, double shear, double inv_pe, double dt, int imex1_estimate,
                     const bie_solve_opts* opts, double* x_out, double* gamma_out, bie_coupled_info* info,
                     void* stream) {
  if (!pq || !xcoef || !gammacoef || !u0 || !lambda || !opts || !x_out || !gamma_out || !info) {
    set_error("null argument");
    return BIE_EINVAL;
  }
  if (x_out == xcoef || gamma_out == gammacoef || !(dt > 0.0) || inv_pe < 0.0) {
    set_error("outputs must not alias the inputs; dt must be positive and 1/Pe non-negative");
    return BIE_EINVAL;
  }
  BIE_TRY(surf_check(ctx, ndrop, p));
  cudaStream_t s = (cudaStream_t)stream;
  std::memset(info, 0, sizeof(*info));
  info->err_imex1 = -1.0;
  SurfLayout L, L0;
  BIE_TRY(surf_layout(ctx, ndrop, p, true, L));
  BIE_TRY(surf_layout(ctx, ndrop, p, false, L0));
  const long long n = L.nv, ns = L.ns;
  DevBuf<double> f, uinf, b, uh, xh, k0, rhs, gh, fe, fi, du, g1;
  for (DevBuf<double>* v : {&f, &uinf, &b, &uh, &xh, &du}) BIE_TRY(v->alloc(n));
  for (DevBuf<double>* v : {&k0, &rhs, &gh, &fe, &fi, &g1}) BIE_TRY(v->alloc(ns));
  const int rprec = (opts->precision & 0xff) == BIE_FP64 ? BIE_FP64 : opts->residual_precision;
  std::vector<double> m0(ndrop), m1(ndrop), ax(ndrop), ad(ndrop);
  BIE_TRY(surf_integrals(L, xcoef, gammacoef, 1, m0.data(), s));
  auto axpby = [&](double a, const double* xv, double bcoef, double* yv, long long len) -> int {
    k_axpby<<<nblk(len), 256, 0, s>>>(a, xv, bcoef, yv, len);
    count_launch();
    BIE_CUDA_TRY(cudaGetLastError());
    return BIE_OK;
  };
  // u^t at (x^t, Gamma^t) unless the caller holds it from a rejected attempt
  if (!u0_valid) {
    BIE_TRY(velocity_solve(ctx, ndrop, p, pq, L.voff, n, xcoef, gammacoef, elasticity, x_s, lambda, shear, opts,
                           rprec, f.ptr, uinf.ptr, b.ptr, u0, &info->solve[0], stream));
    info->velocity_solves++;
  }
  // x^{t+dt/2} = x^t + (dt/2) u^t
  BIE_CUDA_TRY(cudaMemcpyAsync(xh.ptr, xcoef, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  BIE_TRY(axpby(0.5 * dt, u0, 1.0, xh.ptr, n));
  // Gamma^{t+dt/2}: (I - (dt/2) (1/Pe) lap_{x^{t+dt/2}}) Gamma_h = Gamma^t + (dt/2) f_E(x^t, u^t, Gamma^t)
  BIE_TRY(surf_rates(L, xcoef, u0, gammacoef, 0.0, k0.ptr, nullptr, s));
  BIE_CUDA_TRY(cudaMemcpyAsync(rhs.ptr, gammacoef, ns * sizeof(double), cudaMemcpyDeviceToDevice, s));
  BIE_TRY(axpby(0.5 * dt, k0.ptr, 1.0, rhs.ptr, ns));
  BIE_TRY(surf_implicit_solve(L, xh.ptr, rhs.ptr, 0.5 * dt * inv_pe, gh.ptr, 1e-13, &info->implicit_iterations, s));
  // u^{t+dt/2} at (x^{t+dt/2}, Gamma^{t+dt/2})
  BIE_TRY(velocity_solve(ctx, ndrop, p, pq, L.voff, n, xh.ptr, gh.ptr, elasticity, x_s, lambda, shear, opts, rprec,
                         f.ptr, uinf.ptr, b.ptr, uh.ptr, &info->solve[1], stream));
  info->velocity_solves++;
  // x^{t+dt} = x^t + dt u^{t+dt/2};  Gamma^{t+dt} = Gamma^t + dt (f_E + f_I)(x^{t+dt/2}, u^{t+dt/2}, Gamma_h)
  BIE_CUDA_TRY(cudaMemcpyAsync(x_out, xcoef, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  BIE_TRY(axpby(dt, uh.ptr, 1.0, x_out, n));
  BIE_TRY(surf_rates(L, xh.ptr, uh.ptr, gh.ptr, inv_pe, fe.ptr, fi.ptr, s));
  BIE_CUDA_TRY(cudaMemcpyAsync(gamma_out, gammacoef, ns * sizeof(double), cudaMemcpyDeviceToDevice, s));
  BIE_TRY(axpby(dt, fe.ptr, 1.0, gamma_out, ns));
  BIE_TRY(axpby(dt, fi.ptr, 1.0, gamma_out, ns));
  // error estimates of Alg. 1
  BIE_CUDA_TRY(cudaMemcpyAsync(du.ptr, uh.ptr, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  BIE_TRY(axpby(-dt, u0, dt, du.ptr, n));
  BIE_TRY(surf_absmax(L0, du.ptr, 3, ad.data(), s));
  BIE_TRY(surf_absmax(L0, x_out, 3, ax.data(), s));
  BIE_TRY(surf_integrals(L, x_out, gamma_out, 1, m1.data(), s));
  for (int d = 0; d < ndrop; ++d) {
    info->err_drop = std::max(info->err_drop, ad[d] / ax[d]);
    info->err_conservation = std::max(info->err_conservation, std::fabs(m1[d] - m0[d]) / std::fabs(m0[d]));
  }
  if (imex1_estimate) {
    // Gamma_IMEX1: (I - dt (1/Pe) lap_{x^{t+dt}}) G1 = Gamma^t + dt f_E(x^t, u^t, Gamma^t)
    BIE_CUDA_TRY(cudaMemcpyAsync(rhs.ptr, gammacoef, ns * sizeof(double), cudaMemcpyDeviceToDevice, s));
    BIE_TRY(axpby(dt, k0.ptr, 1.0, rhs.ptr, ns));
    int it1 = 0;
    BIE_TRY(surf_implicit_solve(L, x_out, rhs.ptr, dt * inv_pe, g1.ptr, 1e-13, &it1, s));
    BIE_TRY(axpby(1.0, gamma_out, -1.0, g1.ptr, ns));
    std::vector<double> ag(ndrop), an(ndrop);
    BIE_TRY(surf_absmax(L0, g1.ptr, 1, ag.data(), s));
    BIE_TRY(surf_absmax(L0, gamma_out, 1, an.data(), s));
    info->err_imex1 = 0.0;
    for (int d = 0; d < ndrop; ++d) info->err_imex1 = std::max(info->err_imex1, ag[d] / an[d]);
  }
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  return BIE_OK;
}

void bie_reparam_opts_default(bie_reparam_opts* o) {
  if (!o) return;
  o->u_rep = 2;
  o->p_cutoff = 0.05;
  o->smooth = 0;
  o->dtau = 0.5;
  o->eps = 1e-10;
  o->max_iter = 200;
}

}  // extern "C"

namespace bie {

// Alg. 2 for one degree group: drops `drops` of degree p, coefficients at voff[d] (shape) and
// soff[d] (surfactant) in the caller's arrays.
static int reparam_group(bie_ctx* ctx, int p, const std::vector<int>& drops, const std::vector<long long>& voff,
                         const std::vector<long long>& soff, double* xcoef, double* gammacoef,
                         const bie_reparam_opts* o, bie_reparam_info* info, cudaStream_t s) {
  const int P = o->u_rep * (p + 1) - 1;
  const long long nd = (long long)drops.size();
  const long long N = ngrid(P), nC = ncoef(P);
  Plan *plP, *plp;
  BIE_TRY(get_plan(ctx, P, P, &plP));  // synthesis of the energy gradient, analysis at degree P
  BIE_TRY(get_plan(ctx, p, P, &plp));  // the final analysis to degree p
  // recursion coefficients (a, b) of the normalised associated Legendre functions, rows of order m
  std::vector<double> ab(2 * (size_t)(P + 1) * (P + 2) / 2, 0.0);
  for (int m = 0; m <= P; ++m)
    for (int n = m + 2; n <= P; ++n) {
      const long long r = 2 * ((long long)m * (P + 1) - (long long)m * (m - 1) / 2 + (n - m));
      ab[r] = std::sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
      ab[r + 1] = -std::sqrt(((double)(n - 1) * (n - 1) - (double)m * m) / (4.0 * (n - 1) * (n - 1) - 1.0));
    }
  std::vector<double> tn, wn;
  gauss_legendre(P + 1, tn, wn);
  std::vector<long long> vo, so, vof, sof;
  for (int d : drops) {
    vo.push_back(voff[d]);
    so.push_back(soff[d]);
    for (int c = 0; c < 3; ++c) vof.push_back(voff[d] + c * ncoef(p));
    sof.push_back(soff[d]);
  }
  DevBuf<double> dab, dnodes, x0, xt, sc, th, ph, E, gradE, gv, gmax, H, F, a_d, norms, gE;
  DevBuf<long long> dvo, dso, dvof, dsof;
  DevBuf<int> active;
  BIE_TRY(dab.upload(ab));
  BIE_TRY(dnodes.upload(tn));
  BIE_TRY(dvo.upload(vo));
  BIE_TRY(dso.upload(so));
  BIE_TRY(dvof.upload(vof));
  BIE_TRY(dsof.upload(sof));
  for (DevBuf<double>* b : {&x0, &xt, &sc}) BIE_TRY(b->alloc(nd * 3 * nC));
  for (DevBuf<double>* b : {&th, &ph}) BIE_TRY(b->alloc(nd * N));
  BIE_TRY(E.alloc(nd * 9 * N));
  for (DevBuf<double>* b : {&gradE, &gv}) BIE_TRY(b->alloc(nd * 3 * N));
  BIE_TRY(gmax.alloc(nd));
  BIE_TRY(H.alloc(nd * 3 * (P + 1) * (size_t)(P + 1) * 2));
  BIE_TRY(F.alloc(nd * 3 * (P + 1) * (size_t)(P + 1) * 2));
  BIE_TRY(a_d.alloc(nd * (P + 1)));
  BIE_TRY(norms.alloc(nd * (P + 1) * 2));
  BIE_TRY(active.alloc(nd));
  // x~ = x0 = the shape zero-padded to degree P; the angles start at the grid points
  BIE_TRY(launch_pad_coef(xcoef, dvo.ptr, p, P, nd, 3, x0.ptr, s));
  BIE_CUDA_TRY(cudaMemcpyAsync(xt.ptr, x0.ptr, nd * 3 * nC * sizeof(double), cudaMemcpyDeviceToDevice, s));
  BIE_TRY(launch_grid_points(dnodes.ptr, P, nd, th.ptr, ph.ptr, s));
  BIE_TRY(launch_eval_points(x0.ptr, 3, P, nd, N, th.ptr, ph.ptr, dab.ptr, 1, E.ptr, s));
  std::vector<int> act(nd, 1), steps(nd, 0);
  std::vector<double> nrm(nd * (P + 1) * 2), av(nd * (P + 1)), gm(nd, 0.0), en(nd, 0.0);
  for (int it = 0; it < o->max_iter; ++it) {
    // adaptive cutoff (Eq. ncutoff_adaptive) and attenuation per drop, from the current x~
    BIE_TRY(launch_mode_norms(xt.ptr, P, nd, norms.ptr, s));
    BIE_CUDA_TRY(cudaMemcpyAsync(nrm.data(), norms.ptr, nrm.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    BIE_CUDA_TRY(cudaStreamSynchronize(s));
    for (long long d = 0; d < nd; ++d) {
      const double* nd_ = nrm.data() + d * (P + 1) * 2;
      double n1 = 0.0;
      for (int n = 1; n <= P; ++n) n1 += nd_[2 * n];
      int ncut = P;
      double tail = n1;  // sum over n >= l of the per-degree norm sums
      for (int l = 2; l <= P; ++l) {
        tail -= nd_[2 * (l - 1)];
        if (tail / n1 < o->p_cutoff) {
          ncut = l;
          break;
        }
      }
      double e = 0.0;
      for (int n = 0; n <= P; ++n) {
        const double a = n >= ncut ? (o->smooth ? (double)n / P : 1.0) : 0.0;
        av[d * (P + 1) + n] = a;
        e += a * nd_[2 * n + 1];
      }
      if (it == 0) info->energy_first_max = std::max(info->energy_first_max, e);
      if (act[d]) en[d] = e;
    }
    BIE_CUDA_TRY(cudaMemcpyAsync(a_d.ptr, av.data(), av.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    // grad E = 2 sum_n a_n x~_n^m Y_n^m on the grid (Eq. energy_rep), its tangential part at the points
    BIE_TRY(launch_scale_degrees(xt.ptr, a_d.ptr, P, nd, 3, 2.0, sc.ptr, s));
    BIE_TRY((launch_leg_synth<double, double>(sc.ptr, nullptr, nC, nd * 3, P, plP->T0.ptr, P + 1, H.ptr, 0, s)));
    BIE_TRY((launch_phi_synth<double, double>(H.ptr, nd * 3, P, P, plP->cs.ptr, gradE.ptr, nullptr, N, s)));
    BIE_TRY(launch_rep_gradient(E.ptr, gradE.ptr, N, nd, gv.ptr, gmax.ptr, s));
    BIE_CUDA_TRY(cudaMemcpyAsync(gm.data(), gmax.ptr, nd * sizeof(double), cudaMemcpyDeviceToHost, s));
    BIE_CUDA_TRY(cudaStreamSynchronize(s));
    int nact = 0;
    for (long long d = 0; d < nd; ++d) {
      if (act[d] && !(gm[d] >= o->eps)) act[d] = 0;  // the stopping test of Alg. 2 (NaN stops too)
      nact += act[d];
    }
    if (!nact) break;
    // forward Euler step of the angles, then the original expansion at the new angles analysed on the
    // grid (Eq. rep_trasf1)
    BIE_CUDA_TRY(cudaMemcpyAsync(active.ptr, act.data(), nd * sizeof(int), cudaMemcpyHostToDevice, s));
    BIE_TRY(launch_rep_step(E.ptr, gv.ptr, N, nd, active.ptr, o->dtau, th.ptr, ph.ptr, s));
    for (long long d = 0; d < nd; ++d) steps[d] += act[d];
    BIE_TRY(launch_eval_points(x0.ptr, 3, P, nd, N, th.ptr, ph.ptr, dab.ptr, 1, E.ptr, s));
    BIE_TRY(launch_analyze(E.ptr, nullptr, 3 * N, nd * 3, P, P, plP->cs.ptr, plP->A.ptr, F.ptr, xt.ptr, nullptr, nC,
                           s));
  }
  for (long long d = 0; d < nd; ++d) {
    info->iterations = std::max(info->iterations, steps[d]);
    info->converged += act[d] ? 0 : 1;
    info->g_max = std::max(info->g_max, gm[d]);
    info->energy_last_max = std::max(info->energy_last_max, en[d]);
  }
  // Eq. rep_trasf2: the surfactant at the final angles; shape and surfactant analysed to degree p
  BIE_TRY(launch_analyze(E.ptr, nullptr, 3 * N, nd * 3, P, p, plp->cs.ptr, plp->A.ptr, F.ptr, xcoef, dvof.ptr, 0, s));
  if (gammacoef) {
    BIE_TRY(launch_pad_coef(gammacoef, dso.ptr, p, P, nd, 1, x0.ptr, s));
    BIE_TRY(gE.alloc(nd * N));
    BIE_TRY(launch_eval_points(x0.ptr, 1, P, nd, N, th.ptr, ph.ptr, dab.ptr, 0, gE.ptr, s));
    BIE_TRY(launch_analyze(gE.ptr, nullptr, N, nd, P, p, plp->cs.ptr, plp->A.ptr, F.ptr, gammacoef, dsof.ptr, 0, s));
  }
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  return BIE_OK;
}

}  // namespace bie

extern "C" {

int bie_reparametrize(bie_ctx* ctx, int ndrop, const int* p, double* xcoef, double* gammacoef,
                      const bie_reparam_opts* opts, bie_reparam_info* info, void* stream) {
  if (!ctx || !p || !xcoef || !opts || !info || ndrop <= 0) {
    set_error("bie_reparametrize: null or empty argument");
    return BIE_EINVAL;
  }
  if (opts->u_rep < 1 || !(opts->p_cutoff > 0.0 && opts->p_cutoff < 1.0) || !(opts->dtau > 0.0) ||
      !(opts->eps > 0.0) || opts->max_iter < 0) {
    set_error("bie_reparametrize: need u_rep >= 1, 0 < p_cutoff < 1, dtau > 0, eps > 0, max_iter >= 0");
    return BIE_EINVAL;
  }
  BIE_TRY(check_degrees(ndrop, p));
  for (int d = 0; d < ndrop; ++d)
    if (opts->u_rep * (p[d] + 1) - 1 > 4 * BIE_MAX_P) {
      set_error("bie_reparametrize: working degree u_rep (p+1) - 1 above 4 BIE_MAX_P");
      return BIE_EINVAL;
    }
  if (ndrop > 65535) {
    set_error("bie_reparametrize: at most 65535 drops per call");
    return BIE_EINVAL;
  }
  BIE_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  std::memset(info, 0, sizeof(*info));
  Phase ph(ctx, "reparametrize", s);
  std::vector<long long> voff(ndrop), soff(ndrop);
  std::map<int, std::vector<int>> byp;
  long long v = 0, g = 0;
  for (int d = 0; d < ndrop; ++d) {
    voff[d] = v;
    soff[d] = g;
    v += 3 * ncoef(p[d]);
    g += ncoef(p[d]);
    byp[p[d]].push_back(d);
  }
  for (auto& kv : byp) BIE_TRY(reparam_group(ctx, kv.first, kv.second, voff, soff, xcoef, gammacoef, opts, info, s));
  return BIE_OK;
}

double bie_next_dt(double dt, double err, double tol, double dt_max) {
  if (!(err > 0.0)) return dt_max;
  return std::min(dt_max, dt * std::sqrt(0.9 * tol / err));
}

int bie_run_coupled(bie_ctx* ctx, int ndrop, const int* p, const int* pq, double* xcoef, double* gammacoef,
                    double elasticity, double x_s, const double* lambda, double shear, double inv_pe, double T,
                    double dt0, double tol, double dt_max, int estimator, int max_steps, const bie_solve_opts* opts,
                    const bie_reparam_opts* reparam, bie_run_info* info, void* stream) {
  if (!ctx || !p || !xcoef || !gammacoef || !info || !(T > 0.0) || !(dt0 > 0.0) || !(tol > 0.0) ||
      !(dt_max > 0.0) || max_steps < 1 || (estimator != BIE_ERR_CONSERVATION && estimator != BIE_ERR_IMEX1)) {
    set_error("null argument or bad run parameters");
    return BIE_EINVAL;
  }
  BIE_TRY(surf_check(ctx, ndrop, p));
  cudaStream_t s = (cudaStream_t)stream;
  std::memset(info, 0, sizeof(*info));
  long long n = 0, ns = 0;
  for (int d = 0; d < ndrop; ++d) {
    n += 3 * ncoef(p[d]);
    ns += ncoef(p[d]);
  }
  DevBuf<double> u0, x1, g1;
  BIE_TRY(u0.alloc(n));
  BIE_TRY(x1.alloc(n));
  BIE_TRY(g1.alloc(ns));
  double t = 0.0, dt = std::min(dt0, dt_max);
  int u0_valid = 0;
  for (int k = 0; k < max_steps && t < T * (1.0 - 1e-14); ++k) {
    const double h = std::min(dt, T - t);
    bie_coupled_info ci;
    BIE_TRY(bie_step_coupled(ctx, ndrop, p, pq, xcoef, gammacoef, u0.ptr, u0_valid, elasticity, x_s, lambda, shear,
                             inv_pe, h, estimator == BIE_ERR_IMEX1, opts, x1.ptr, g1.ptr, &ci, stream));
    info->velocity_solves += ci.velocity_solves;
    u0_valid = 1;
    const double es = estimator == BIE_ERR_IMEX1 ? ci.err_imex1 : ci.err_conservation;
    const double err = std::max(ci.err_drop, es);
    if (err < tol) {
      t += h;
      BIE_CUDA_TRY(cudaMemcpyAsync(xcoef, x1.ptr, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      BIE_CUDA_TRY(cudaMemcpyAsync(gammacoef, g1.ptr, ns * sizeof(double), cudaMemcpyDeviceToDevice, s));
      u0_valid = 0;
      info->steps_accepted++;
      info->err_max_accepted = std::max(info->err_max_accepted, err);
      if (reparam) {  // Alg. 2 after every kept step
        bie_reparam_info ri;
        BIE_TRY(bie_reparametrize(ctx, ndrop, p, xcoef, gammacoef, reparam, &ri, stream));
        info->reparam_iterations += ri.iterations;
      }
    } else {
      info->steps_rejected++;
    }
    dt = bie_next_dt(h, err, tol, dt_max);
  }
  BIE_CUDA_TRY(cudaStreamSynchronize(s));
  info->t = t;
  info->dt_next = dt;
  if (t < T * (1.0 - 1e-14)) {
    set_error("bie_run_coupled: max_steps reached before T");
    return BIE_ENOCONV;
  }
  return BIE_OK;
}

long long bie_launch_count(void) { return g_launches.load(); }

long long bie_debug_table(int which, int a, int b, int c, double x, double* out, long long cap) {
  std::vector<double> v;
  if (which == 0) {
    if (a < 0 || a > 4 * BIE_MAX_P) return -1;
    std::vector<double> t, w;
    gauss_legendre(a + 1, t, w);
    v = t;
    v.insert(v.end(), w.begin(), w.end());
  } else if (which == 1) {
    if (a < 0 || a > BIE_MAX_P || c < a || c > 4 * BIE_MAX_P || b < 0 || b > 2) return -1;
    legendre_table(a, c, b, v);
  } else if (which == 2) {
    if (a < 0 || a > 2 * BIE_MAX_P) return -1;
    v.resize((size_t)(2 * a + 1) * (2 * a + 1));
    wigner_small_d(a, x, v.data());
  } else if (which == 3) {
    if (a < 0 || a > 4 * BIE_MAX_P) return -1;
    singular_weights(a, v);
  } else {
    return -1;
  }
  if (out) std::memcpy(out, v.data(), sizeof(double) * std::min<long long>(cap, (long long)v.size()));
  return (long long)v.size();
}

}  // extern "C"
