// Grouped batch engine: one CN step of many independent problems (Sec. 2's
// scheme on each; sizes, orders and coefficients may differ) advanced with one
// launch per stage for the whole batch.
//
// Every stage of the single-problem solve -- each FFT or direct-sum pass of
// the Toeplitz products, each transpose, smoothing, transfer, the one-launch
// tail of the V-cycle, the Krylov matvec, each Gram-Schmidt pass, the Givens
// update -- runs as one grouped launch over a work list of (problem, unit)
// items (kernels_*.cu, GItem / GGate).  The problems' FGMRES iterations run
// in lockstep: iteration j of every problem that is still iterating is one
// sequence of grouped launches, and a problem whose residual estimate met its
// tolerance (or its restart length) closes its gate on the device, so the
// later launches skip it.  One restart cycle of the whole batch -- right-hand
// side, norms, the restart length's iterations, the solution update and the
// true residual -- is therefore a fixed sequence of launches, captured once as
// a CUDA graph and replayed every step; the host reads the per-problem states
// once per cycle.
//
// The engine reuses the problems' handles (fde_create): their multigrid
// hierarchies, spectra, coefficient copies and Krylov workspaces.  It serves
// batches whose problems all use the FP32 V-cycle with structured-Galerkin or
// rediscretised coarse operators, FFT or direct-sum products above a
// one-launch tail, one cycle per preconditioner application, the double-float
// outer apply, one restart length <= 32, and no warm start; other batches run
// on the worker-thread engine (fde_batch.cu).
#include <map>

#include "solver.cuh"

namespace fde {

namespace {

template <typename P>
int dev_alloc(std::vector<void*>& owned, P** out, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(P) + 16) != cudaSuccess) return FDE_ERR_CUDA;
  owned.push_back(q);
  *out = static_cast<P*>(q);
  return FDE_OK;
}

// a device array of records plus its work list
template <typename E>
struct Stage {
  E* ent = nullptr;
  GItem* items = nullptr;
  int nitems = 0;
  int aux = 0;  // max logL (FFT) or max n (direct)
};

template <typename E>
int upload(std::vector<void*>& owned, const std::vector<E>& ents, const std::vector<GItem>& items,
           int aux, Stage<E>* s, cudaStream_t st) {
  s->nitems = (int)items.size();
  s->aux = aux;
  if (ents.empty() || items.empty()) return FDE_OK;
  if (dev_alloc(owned, &s->ent, ents.size()) != FDE_OK) return FDE_ERR_CUDA;
  if (dev_alloc(owned, &s->items, items.size()) != FDE_OK) return FDE_ERR_CUDA;
  if (cudaMemcpyAsync(s->ent, ents.data(), ents.size() * sizeof(E), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(s->items, items.data(), items.size() * sizeof(GItem),
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return FDE_ERR_CUDA;
  return FDE_OK;
}

using FftF = GFftPass<float, float, float>;
using FftDF = GFftPass<double, df, df>;
using Fft32 = GFftPass<double, float, float>;

// one products call of a level (MG::products) for every problem at that level
struct ProductsStage {
  Stage<FftF> fft_rows, fft_cols;
  Stage<GTranspose<float>> tr_in, tr_out;
  Stage<GDirectPass<float>> dir_rows, dir_cols;
};

// the FP64-accurate (double-float) or relaxed (FP32) outer apply of every problem
struct OuterStage {
  Stage<FftDF> rows, cols;
  Stage<GTranspose<double>> tr_in, tr_out;
  Stage<Fft32> rows32, cols32;
  Stage<GTranspose<double>> tr_in32, tr_out32;
};

}  // namespace

struct GroupEngine {
  std::vector<fde_handle*> hs;
  std::vector<MG<float>*> mgs;
  int P = 0, m = 0, maxdepth = 0;
  std::vector<void*> owned;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // [0] restart cycle, [1] first cycle
  long long graph_launches[2] = {0, 0};
  long long launches = 0;
  int *active = nullptr, *incycle = nullptr, *relax = nullptr;
  GSolveState* ss = nullptr;
  GKrylov* kry = nullptr;
  double* scal = nullptr;  // 4 per problem
  std::vector<GSolveState> ss_host;
  std::string err;
  // stages
  Stage<GVec> copy_in, copy_out, rhs_lincomb, norm_b, zero_x, v0_b, v0_r, sub_res, norm_r;
  Stage<GLevelOp<float>> dummy;
  OuterStage outer_old, outer_new_x, outer_new_z[ArnoldiState::kMaxM];
  std::vector<Stage<GVec>> conv_in, conv_out;  // per j: V_j -> b (FP32), x -> Z_j
  // V-cycle: per level, the problems at that level above their tail
  struct LevelStages {
    Stage<GLevelOp<float>> ops;  // records of the level (one per problem)
    std::vector<GItem> fine_items, coarse_items;
    Stage<GLevelOp<float>> fine, coarse;  // items over fine / coarse points
    ProductsStage prod;
    bool any_mass = false;
  };
  std::vector<LevelStages> lvs;
  Stage<GLevelOp<float>> mass_ops[16];
  TailArgs<float>* tails = nullptr;
  int* tail_probs = nullptr;
  int ntail = 0;
  Stage<GKrylov> kry_items;   // items over every problem's Krylov chunks
  double** xs_dev = nullptr;  // solution buffer per problem (update target)
  Stage<GVec> upd_dummy;
  GItem* upd_items = nullptr;
  int upd_nitems = 0;
  GVec *copy_in_host = nullptr, *copy_out_host = nullptr;  // pinned, rewritten every step

  int fail(const char* fmt, ...) {
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    err = buf;
    return FDE_ERR_UNSUPPORTED;
  }

  ~GroupEngine() {
    for (auto g : graph)
      if (g) cudaGraphExecDestroy(g);
    if (cap) cudaStreamDestroy(cap);
    for (void* q : owned) cudaFree(q);
    if (copy_in_host) cudaFreeHost(copy_in_host);
    if (copy_out_host) cudaFreeHost(copy_out_host);
  }

  static bool eligible(fde_handle* h, std::string& why) {
    const fde_params& p = h->p;
    if (p.precision != FDE_PREC_FP32) return why = "precision is not FP32", false;
    if (p.precond != FDE_PRECOND_MG_SG && p.precond != FDE_PRECOND_MG_REDISC)
      return why = "preconditioner is not a Toeplitz V-cycle", false;
    if (p.outer != FDE_OUTER_DF32) return why = "outer apply is not double-float", false;
    if (p.solver != FDE_SOLVER_FGMRES || p.warm != 0) return why = "solver or warm start", false;
    if (p.cycles > 1) return why = "several cycles per application", false;
    if (p.restart > 32) return why = "restart > 32", false;
    auto* mg = dynamic_cast<MG<float>*>(h->mg.get());
    if (!mg) return why = "no FP32 Toeplitz hierarchy", false;
    if (mg->tail0 + 1 >= mg->lv.size() || mg->tail0 == 0) return why = "no one-launch tail", false;
    for (size_t l = 0; l < mg->tail0; ++l)
      if (mg->lv[l].path != FDE_PATH_FFT && mg->lv[l].path != FDE_PATH_DIRECT)
        return why = "a level uses tensor-core products", false;
    return true;
  }

  // ------------------------------------------------------------------ build
  int build(const std::vector<fde_handle*>& handles, cudaStream_t st) {
    hs = handles;
    P = (int)hs.size();
    for (fde_handle* h : hs) {
      std::string why;
      if (!eligible(h, why)) return fail("grouped engine: %s", why.c_str());
      mgs.push_back(static_cast<MG<float>*>(h->mg.get()));
    }
    m = hs[0]->p.restart;
    for (fde_handle* h : hs)
      if (h->p.restart != m) return fail("grouped engine: problems differ in restart length");
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
      return fail("grouped engine: stream creation failed");
    if (dev_alloc(owned, &active, P) || dev_alloc(owned, &incycle, P) ||
        dev_alloc(owned, &relax, P) || dev_alloc(owned, &ss, P) || dev_alloc(owned, &scal, 4 * P))
      return FDE_ERR_CUDA;
    cudaMemsetAsync(relax, 0, P * sizeof(int), st);
    ss_host.resize(P);
    // Krylov records and items over each problem's chunks
    std::vector<GKrylov> kr(P);
    std::vector<GItem> kitems, vitems;
    for (int q = 0; q < P; ++q) {
      fde_handle* h = hs[q];
      GKrylov& e = kr[q];
      e.V = h->V;
      e.Z = h->Z;
      e.ldv = h->ldv;
      e.N = h->N;
      e.part = h->cgs_part;
      e.tickets = h->tickets;
      e.h = h->hdev;
      e.h2 = h->h2dev;
      e.y = h->ydev;
      e.scal = scal + 4 * q;
      e.st = h->ast;
      e.ss = ss + q;
      e.rtol = h->p.rtol;
      e.maxit = h->p.maxit;
      e.relax_on = h->p.relax;
      e.restart = m;
      e.nchunk = (int)(((h->N + 1) / 2 + kGKChunk - 1) / kGKChunk);
      e.prob = q;
      for (int c = 0; c < e.nchunk; ++c) kitems.push_back({q, c});
      const int nv = (int)((h->N + kGChunk - 1) / kGChunk);
      for (int c = 0; c < nv; ++c) vitems.push_back({q, c});
    }
    if (upload(owned, kr, kitems, 0, &kry_items, st)) return FDE_ERR_CUDA;
    kry = kry_items.ent;
    if (dev_alloc(owned, &upd_items, vitems.size())) return FDE_ERR_CUDA;
    cudaMemcpyAsync(upd_items, vitems.data(), vitems.size() * sizeof(GItem), cudaMemcpyHostToDevice,
                    st);
    upd_nitems = (int)vitems.size();
    std::vector<double*> xs(P);
    for (int q = 0; q < P; ++q) xs[q] = hs[q]->hx_out;
    if (dev_alloc(owned, &xs_dev, P)) return FDE_ERR_CUDA;
    cudaMemcpyAsync(xs_dev, xs.data(), P * sizeof(double*), cudaMemcpyHostToDevice, st);

    // vector stages: records per problem, items over kGChunk chunks
    auto vec_stage = [&](Stage<GVec>* s, auto fill) -> int {
      std::vector<GVec> ents(P);
      for (int q = 0; q < P; ++q) {
        GVec e{};
        e.N = hs[q]->N;
        e.prob = q;
        fill(q, hs[q], e);
        ents[q] = e;
      }
      return upload(owned, ents, vitems, 0, s, st);
    };
    // copy-in / copy-out records are rewritten every step from pinned memory
    if (cudaMallocHost(&copy_in_host, 2 * P * sizeof(GVec)) != cudaSuccess ||
        cudaMallocHost(&copy_out_host, P * sizeof(GVec)) != cudaSuccess)
      return FDE_ERR_CUDA;
    {
      std::vector<GItem> cin;
      for (int q = 0; q < P; ++q) {
        const int nv = (int)((hs[q]->N + kGChunk - 1) / kGChunk);
        for (int c = 0; c < nv; ++c) cin.push_back({2 * q, c});
        for (int c = 0; c < nv; ++c) cin.push_back({2 * q + 1, c});
      }
      std::vector<GVec> ents(2 * P);
      for (int q = 0; q < P; ++q) {
        ents[2 * q].N = ents[2 * q + 1].N = hs[q]->N;
        ents[2 * q].prob = ents[2 * q + 1].prob = q;
      }
      if (upload(owned, ents, cin, 0, &copy_in, st)) return FDE_ERR_CUDA;
      std::vector<GVec> eo(P);
      for (int q = 0; q < P; ++q) {
        eo[q].N = hs[q]->N;
        eo[q].prob = q;
      }
      if (upload(owned, eo, vitems, 0, &copy_out, st)) return FDE_ERR_CUDA;
    }
    // b = 2c u - M_old u + 2 h^alpha v  (rhs; tmp holds M_old u)
    if (vec_stage(&rhs_lincomb, [](int, fde_handle* h, GVec& e) {
          e.a = h->hu;
          e.s0 = 2.0 * h->c;
          e.b = h->tmp;
          e.s1 = -1.0;
          e.c = h->hv;
          e.s2 = h->two_h_alpha;
          e.y = h->bwork;
        }))
      return FDE_ERR_CUDA;
    if (vec_stage(&norm_b, [this](int q, fde_handle* h, GVec& e) {
          e.a = h->bwork;
          e.y = scal + 4 * q;  // scal[0] = ||b||
        }))
      return FDE_ERR_CUDA;
    if (vec_stage(&zero_x, [](int, fde_handle* h, GVec& e) { e.y = h->hx_out; }))
      return FDE_ERR_CUDA;
    if (vec_stage(&v0_b, [this](int q, fde_handle* h, GVec& e) {
          e.a = h->bwork;
          e.sptr = scal + 4 * q;
          e.y = h->V;
        }))
      return FDE_ERR_CUDA;
    if (vec_stage(&sub_res, [](int, fde_handle* h, GVec& e) {
          e.a = h->bwork;
          e.b = h->tmp;
          e.y = h->tmp;
        }))
      return FDE_ERR_CUDA;
    if (vec_stage(&norm_r, [this](int q, fde_handle* h, GVec& e) {
          e.a = h->tmp;
          e.y = scal + 4 * q + 1;  // scal[1] = residual norm
        }))
      return FDE_ERR_CUDA;
    if (vec_stage(&v0_r, [this](int q, fde_handle* h, GVec& e) {
          e.a = h->tmp;
          e.sptr = scal + 4 * q + 1;
          e.y = h->V;
        }))
      return FDE_ERR_CUDA;
    conv_in.resize(m);
    conv_out.resize(m);
    for (int j = 0; j < m; ++j) {
      if (vec_stage(&conv_in[j], [&](int q, fde_handle* h, GVec& e) {
            e.a = h->V + (size_t)j * h->ldv;
            e.yf = mgs[q]->lv[0].b;
          }))
        return FDE_ERR_CUDA;
      if (vec_stage(&conv_out[j], [&](int q, fde_handle* h, GVec& e) {
            e.af = mgs[q]->lv[0].x;
            e.y = h->Z + (size_t)j * h->ldv;
          }))
        return FDE_ERR_CUDA;
    }
    // outer applies
    if (build_outer(&outer_old, true, [](fde_handle* h) { return (const double*)h->hu; },
                    [](fde_handle* h) { return h->tmp; }, false, st))
      return FDE_ERR_CUDA;
    if (build_outer(&outer_new_x, false, [](fde_handle* h) { return (const double*)h->hx_out; },
                    [](fde_handle* h) { return h->tmp; }, false, st))
      return FDE_ERR_CUDA;
    for (int j = 0; j < m; ++j)
      if (build_outer(&outer_new_z[j], false,
                      [j](fde_handle* h) { return (const double*)(h->Z + (size_t)j * h->ldv); },
                      [j](fde_handle* h) { return h->V + (size_t)(j + 1) * h->ldv; }, true, st))
        return FDE_ERR_CUDA;
    // V-cycle levels
    for (auto* mg : mgs) maxdepth = std::max(maxdepth, (int)mg->tail0);
    lvs.resize(maxdepth);
    for (int l = 0; l < maxdepth; ++l)
      if (build_level(l, st)) return FDE_ERR_CUDA;
    // tails
    {
      std::vector<TailArgs<float>> ta;
      std::vector<int> tp;
      for (int q = 0; q < P; ++q) {
        ta.push_back(mgs[q]->tail_args(hs[q]));
        tp.push_back(q);
      }
      ntail = P;
      if (dev_alloc(owned, &tails, P) || dev_alloc(owned, &tail_probs, P)) return FDE_ERR_CUDA;
      cudaMemcpyAsync(tails, ta.data(), P * sizeof(TailArgs<float>), cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(tail_probs, tp.data(), P * sizeof(int), cudaMemcpyHostToDevice, st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail("grouped engine: set-up failed");
    return FDE_OK;
  }

  // x -> y with the outer operator of every problem: double-float (want 0
  // when `gated`, else always) and, when gated, the relaxed FP32 variant (want 1)
  template <typename FX, typename FY>
  int build_outer(OuterStage* o, bool old, FX fx, FY fy, bool gated, cudaStream_t st) {
    std::vector<FftDF> r, c;
    std::vector<GTranspose<double>> ti, to;
    std::vector<Fft32> r32, c32;
    std::vector<GTranspose<double>> ti32, to32;
    std::vector<GItem> ir, ic, iti, ito, ir32, ic32, iti32, ito32;
    int mlog = 1, mlog32 = 1;
    for (int q = 0; q < P; ++q) {
      fde_handle* h = hs[q];
      const double* x = fx(h);
      double* y = fy(h);
      df* const* cf = old ? h->cfO : h->cfN;
      df* const* cfT = old ? h->cfOT : h->cfNT;
      const int want = gated ? 0 : -1;
      r.push_back({x, 1, h->n1, h->n2, h->n1, h->logLx, h->S1xd, h->S2xd, h->twxd, cf[0], cf[1],
                   x, h->c, y, 0, q, want});
      c.push_back({h->xT, 1, h->n2, h->n1, h->n2, h->logLy, h->S1yd, h->S2yd, h->twyd, cfT[0],
                   cfT[1], nullptr, 0.0, h->yT, 0, q, want});
      ti.push_back({x, h->n2, h->n1, h->xT, 0, q, want});
      to.push_back({h->yT, h->n1, h->n2, y, 1, q, want});
      mlog = std::max(mlog, std::max(h->logLx, h->logLy));
      const int e = (int)r.size() - 1;
      for (int u = 0; u < (h->n2 + 1) / 2; ++u) ir.push_back({e, u});
      for (int u = 0; u < (h->n1 + 1) / 2; ++u) ic.push_back({e, u});
      const int tiles_in = ((h->n1 + 31) / 32) * ((h->n2 + 31) / 32);
      for (int u = 0; u < tiles_in; ++u) {
        iti.push_back({e, u});
        ito.push_back({e, u});
      }
      if (gated && h->p.relax) {
        r32.push_back({x, 1, h->n1, h->n2, h->n1, h->logLx, h->S1x32, h->S2x32, h->twx32,
                       h->cf32[0], h->cf32[1], x, h->c, y, 0, q, 1});
        c32.push_back({h->xT, 1, h->n2, h->n1, h->n2, h->logLy, h->S1y32, h->S2y32, h->twy32,
                       h->cf32T[0], h->cf32T[1], nullptr, 0.0, h->yT, 0, q, 1});
        ti32.push_back({x, h->n2, h->n1, h->xT, 0, q, 1});
        to32.push_back({h->yT, h->n1, h->n2, y, 1, q, 1});
        mlog32 = std::max(mlog32, std::max(h->logLx, h->logLy));
        const int e2 = (int)r32.size() - 1;
        for (int u = 0; u < (h->n2 + 1) / 2; ++u) ir32.push_back({e2, u});
        for (int u = 0; u < (h->n1 + 1) / 2; ++u) ic32.push_back({e2, u});
        for (int u = 0; u < tiles_in; ++u) {
          iti32.push_back({e2, u});
          ito32.push_back({e2, u});
        }
      }
    }
    if (upload(owned, r, ir, mlog, &o->rows, st) || upload(owned, c, ic, mlog, &o->cols, st) ||
        upload(owned, ti, iti, 0, &o->tr_in, st) || upload(owned, to, ito, 0, &o->tr_out, st) ||
        upload(owned, r32, ir32, mlog32, &o->rows32, st) ||
        upload(owned, c32, ic32, mlog32, &o->cols32, st) ||
        upload(owned, ti32, iti32, 0, &o->tr_in32, st) ||
        upload(owned, to32, ito32, 0, &o->tr_out32, st))
      return FDE_ERR_CUDA;
    return FDE_OK;
  }

  int build_level(int l, cudaStream_t st) {
    LevelStages& S = lvs[l];
    std::vector<GLevelOp<float>> ops;
    std::vector<GItem> fine, coarse;
    std::vector<FftF> fr, fc;
    std::vector<GTranspose<float>> ti, to;
    std::vector<GDirectPass<float>> dr, dc;
    std::vector<GItem> ifr, ifc, iti, ito, idr, idc;
    int mlog = 1, maxn = 1;
    for (int q = 0; q < P; ++q) {
      MG<float>* mg = mgs[q];
      if (l >= (int)mg->tail0) continue;
      fde_handle* h = hs[q];
      auto& L = mg->lv[l];
      auto& C = mg->lv[l + 1];
      const bool mass = mg->sg && l > 0;
      GLevelOp<float> e{};
      e.n1 = L.n1;
      e.n2 = L.n2;
      e.x = L.x;
      e.b = L.b;
      e.kx = L.kx;
      e.W = L.W;
      e.xby = L.xby;
      e.xbx = L.xbx;
      e.mass = L.mass;
      e.bx0 = (float)L.bx0;
      e.bx1 = (float)L.bx1;
      e.by0 = (float)L.by0;
      e.by1 = (float)L.by1;
      e.c = (float)h->c;
      e.bc = C.b;
      e.xc = C.x;
      e.rscale = (float)mg->rscale;
      e.prob = q;
      ops.push_back(e);
      const int ei = (int)ops.size() - 1;
      if (mass) S.any_mass = true;
      for (int c = 0; c < (int)((L.N + kGChunk - 1) / kGChunk); ++c) fine.push_back({ei, c});
      const size_t NC = (size_t)coarse_n(L.n1) * coarse_n(L.n2);
      for (int c = 0; c < (int)((NC + kGChunk - 1) / kGChunk); ++c) coarse.push_back({ei, c});
      // products (MG::products): x-operand xby on structured-Galerkin levels
      const float* xin_x = mass ? L.xby : L.x;
      const float* xin_y = mass ? L.xbx : L.x;
      const float* M = mass ? L.mass : L.x;
      const double cm = mass ? 1.0 : h->c;
      if (L.path == FDE_PATH_FFT) {
        fr.push_back({xin_x, 1, L.n1, L.n2, L.n1, L.logLx, L.S1x, L.S2x, L.twx, L.dp, L.dm, M, cm,
                      L.kx, 0, q, -1});
        fc.push_back({L.xT, 1, L.n2, L.n1, L.n2, L.logLy, L.S1y, L.S2y, L.twy, L.epT, L.emT,
                      nullptr, 0.0, L.yT, 0, q, -1});
        ti.push_back({xin_y, L.n2, L.n1, L.xT, 0, q, -1});
        to.push_back({L.yT, L.n1, L.n2, L.kx, 1, q, -1});
        mlog = std::max(mlog, std::max(L.logLx, L.logLy));
        const int f = (int)fr.size() - 1;
        for (int u = 0; u < (L.n2 + 1) / 2; ++u) ifr.push_back({f, u});
        for (int u = 0; u < (L.n1 + 1) / 2; ++u) ifc.push_back({f, u});
        const int tiles = ((L.n1 + 31) / 32) * ((L.n2 + 31) / 32);
        for (int u = 0; u < tiles; ++u) {
          iti.push_back({f, u});
          ito.push_back({f, u});
        }
      } else {
        dr.push_back({xin_x, 1, L.n1, L.n2, L.n1, L.txT, L.dp, L.dm, M, cm, L.kx, 0, q, -1});
        dc.push_back({xin_y, L.n1, 1, L.n1, L.n2, L.tyT, L.ep, L.em, nullptr, 0.0, L.kx, 1, q, -1});
        maxn = std::max(maxn, std::max(L.n1, L.n2));
        const int d = (int)dr.size() - 1;
        for (int u = 0; u < L.n2; ++u) idr.push_back({d, u});
        for (int u = 0; u < L.n1; ++u) idc.push_back({d, u});
      }
    }
    if (upload(owned, ops, fine, 0, &S.fine, st)) return FDE_ERR_CUDA;
    S.coarse = S.fine;  // same records, coarse-grid items
    S.coarse.items = nullptr;
    S.coarse.nitems = (int)coarse.size();
    if (!coarse.empty()) {
      if (dev_alloc(owned, &S.coarse.items, coarse.size())) return FDE_ERR_CUDA;
      cudaMemcpyAsync(S.coarse.items, coarse.data(), coarse.size() * sizeof(GItem),
                      cudaMemcpyHostToDevice, st);
    }
    ProductsStage& pr = S.prod;
    if (upload(owned, fr, ifr, mlog, &pr.fft_rows, st) ||
        upload(owned, fc, ifc, mlog, &pr.fft_cols, st) ||
        upload(owned, ti, iti, 0, &pr.tr_in, st) || upload(owned, to, ito, 0, &pr.tr_out, st) ||
        upload(owned, dr, idr, maxn, &pr.dir_rows, st) ||
        upload(owned, dc, idc, maxn, &pr.dir_cols, st))
      return FDE_ERR_CUDA;
    // the mass pre-pass runs on the structured-Galerkin levels > 0 only: the
    // records of level 0 (or of a rediscretised hierarchy) skip it below
    return FDE_OK;
  }

  // ------------------------------------------------------------------ stages
#define GCHK(call)                                     \
  do {                                                 \
    cudaError_t _e = (call);                           \
    ++launches;                                        \
    if (_e != cudaSuccess) return FDE_ERR_CUDA;        \
  } while (0)

  int run_outer(const OuterStage& o, GGate g, cudaStream_t st) {
    GCHK(launch_g_fft_pass(o.rows.ent, o.rows.items, o.rows.nitems, o.rows.aux, g, st));
    GCHK(launch_g_transpose(o.tr_in.ent, o.tr_in.items, o.tr_in.nitems, g, st));
    GCHK(launch_g_fft_pass(o.cols.ent, o.cols.items, o.cols.nitems, o.cols.aux, g, st));
    GCHK(launch_g_transpose(o.tr_out.ent, o.tr_out.items, o.tr_out.nitems, g, st));
    if (o.rows32.nitems) {
      GCHK(launch_g_fft_pass(o.rows32.ent, o.rows32.items, o.rows32.nitems, o.rows32.aux, g, st));
      GCHK(launch_g_transpose(o.tr_in32.ent, o.tr_in32.items, o.tr_in32.nitems, g, st));
      GCHK(launch_g_fft_pass(o.cols32.ent, o.cols32.items, o.cols32.nitems, o.cols32.aux, g, st));
      GCHK(launch_g_transpose(o.tr_out32.ent, o.tr_out32.items, o.tr_out32.nitems, g, st));
    }
    return FDE_OK;
  }

  int run_products(int l, GGate g, cudaStream_t st) {
    LevelStages& S = lvs[l];
    const ProductsStage& p = S.prod;
    if (S.any_mass) GCHK(launch_g_level_op(G_MASS, S.fine.ent, S.fine.items, S.fine.nitems, g, st));
    GCHK(launch_g_fft_pass(p.fft_rows.ent, p.fft_rows.items, p.fft_rows.nitems, p.fft_rows.aux, g,
                           st));
    GCHK(launch_g_direct_pass(p.dir_rows.ent, p.dir_rows.items, p.dir_rows.nitems, p.dir_rows.aux,
                              g, st));
    GCHK(launch_g_transpose(p.tr_in.ent, p.tr_in.items, p.tr_in.nitems, g, st));
    GCHK(launch_g_fft_pass(p.fft_cols.ent, p.fft_cols.items, p.fft_cols.nitems, p.fft_cols.aux, g,
                           st));
    GCHK(launch_g_direct_pass(p.dir_cols.ent, p.dir_cols.items, p.dir_cols.nitems, p.dir_cols.aux,
                              g, st));
    GCHK(launch_g_transpose(p.tr_out.ent, p.tr_out.items, p.tr_out.nitems, g, st));
    return FDE_OK;
  }

  // one V-cycle of every active problem (MG::cycle, level by level)
  int run_vcycle(GGate g, cudaStream_t st) {
    const int nu_pre = hs[0]->p.nu_pre, nu_post = hs[0]->p.nu_post;
    for (int l = 0; l < maxdepth; ++l) {
      LevelStages& S = lvs[l];
      if (nu_pre >= 1) GCHK(launch_g_level_op(G_MUL, S.fine.ent, S.fine.items, S.fine.nitems, g, st));
      for (int s = 1; s < nu_pre; ++s) {
        if (int r = run_products(l, g, st)) return r;
        GCHK(launch_g_level_op(G_SMOOTH, S.fine.ent, S.fine.items, S.fine.nitems, g, st));
      }
      if (int r = run_products(l, g, st)) return r;
      GCHK(launch_g_level_op(G_RESID, S.fine.ent, S.fine.items, S.fine.nitems, g, st));
      GCHK(launch_g_level_op(G_RESTRICT, S.coarse.ent, S.coarse.items, S.coarse.nitems, g, st));
    }
    GCHK(launch_g_mg_tail(tails, tail_probs, ntail, g, st));
    for (int l = maxdepth - 1; l >= 0; --l) {
      LevelStages& S = lvs[l];
      GCHK(launch_g_level_op(G_PROLONG, S.fine.ent, S.fine.items, S.fine.nitems, g, st));
      for (int s = 0; s < nu_post; ++s) {
        if (int r = run_products(l, g, st)) return r;
        GCHK(launch_g_level_op(G_SMOOTH, S.fine.ent, S.fine.items, S.fine.nitems, g, st));
      }
    }
    return FDE_OK;
  }

  // one restart cycle of the whole batch; first: preceded by the right-hand
  // side, ||b||, x = 0 and V_0 = b / ||b||; else V_0 = r / ||r||
  int run_cycle(bool first, cudaStream_t st) {
    GGate ga{active, relax}, gc{incycle, relax};
    if (first) {
      GGate all{incycle, relax};
      // every problem takes part in the right-hand side (incycle = 1 here)
      if (int r = run_outer(outer_old, all, st)) return r;
      GCHK(launch_g_vec(GV_LINCOMB, rhs_lincomb.ent, rhs_lincomb.items, rhs_lincomb.nitems, all,
                        st));
      GCHK(launch_g_norm(norm_b.ent, kry, norm_b.items, norm_b.nitems, all, st));
      GCHK(launch_g_vec(GV_ZERO, zero_x.ent, zero_x.items, zero_x.nitems, all, st));
      GCHK(launch_g_solve_start(kry, P, active, incycle, st));
      GCHK(launch_g_vec(GV_SCALE_INV, v0_b.ent, v0_b.items, v0_b.nitems, gc, st));
    } else {
      GCHK(launch_g_vec(GV_SCALE_INV, v0_r.ent, v0_r.items, v0_r.nitems, gc, st));
    }
    GCHK(launch_g_cycle_start(kry, P, first ? 1 : 0, incycle, active, relax, st));
    for (int j = 0; j < m; ++j) {
      GCHK(launch_g_vec(GV_D2F, conv_in[j].ent, conv_in[j].items, conv_in[j].nitems, ga, st));
      if (int r = run_vcycle(ga, st)) return r;
      GCHK(launch_g_vec(GV_F2D, conv_out[j].ent, conv_out[j].items, conv_out[j].nitems, ga, st));
      if (int r = run_outer(outer_new_z[j], ga, st)) return r;
      GCHK(launch_g_cgs2(kry, kry_items.items, kry_items.nitems, j, ga, active, relax, st));
      launches += 3;
    }
    GCHK(launch_g_lsq(kry, P, incycle, st));
    GCHK(launch_g_update(kry, xs_dev, upd_items, upd_nitems, incycle, st));
    if (int r = run_outer(outer_new_x, gc, st)) return r;
    GCHK(launch_g_vec(GV_SUB, sub_res.ent, sub_res.items, sub_res.nitems, gc, st));
    GCHK(launch_g_norm(norm_r.ent, kry, norm_r.items, norm_r.nitems, gc, st));
    GCHK(launch_g_cycle_end(kry, P, incycle, st));
    return FDE_OK;
  }

  int capture(int first) {
    const long long l0 = launches;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return fail("grouped engine: stream capture failed");
    const int rc = run_cycle(first != 0, cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cap, &g);
    graph_launches[first] = launches - l0;
    launches = l0;
    if (rc != FDE_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return fail("grouped engine: capture of the cycle failed");
    }
    const cudaError_t ei = cudaGraphInstantiate(&graph[first], g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return fail("grouped engine: graph instantiation failed");
    return FDE_OK;
  }

  // one CN step of every problem
  int step(const double* const* u_prev, const double* const* v_half, double* const* u_next,
           cudaStream_t st, std::vector<int>& rc, fde_stats* stats) {
    if (!graph[1] && capture(1)) return FDE_ERR_UNSUPPORTED;
    if (!graph[0] && capture(0)) return FDE_ERR_UNSUPPORTED;
    // inputs into the handles' fixed buffers (the graph reads those)
    for (int q = 0; q < P; ++q) {
      GVec& a = copy_in_host[2 * q];
      GVec& b = copy_in_host[2 * q + 1];
      a = GVec{};
      b = GVec{};
      a.a = u_prev[q];
      a.y = hs[q]->hu;
      b.a = v_half[q];
      b.y = hs[q]->hv;
      a.N = b.N = hs[q]->N;
      a.prob = b.prob = q;
      GVec& o = copy_out_host[q];
      o = GVec{};
      o.a = hs[q]->hx_out;
      o.y = u_next[q];
      o.N = hs[q]->N;
      o.prob = q;
    }
    std::vector<int> ones(P, 1);
    if (cudaMemcpyAsync(copy_in.ent, copy_in_host, 2 * P * sizeof(GVec), cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(copy_out.ent, copy_out_host, P * sizeof(GVec), cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(incycle, ones.data(), P * sizeof(int), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
      return FDE_ERR_CUDA;
    GGate all{incycle, relax};
    GCHK(launch_g_vec(GV_COPY, copy_in.ent, copy_in.items, copy_in.nitems, all, st));
    if (cudaGraphLaunch(graph[1], st) != cudaSuccess) return FDE_ERR_CUDA;
    launches += graph_launches[1];
    for (;;) {
      if (cudaMemcpyAsync(ss_host.data(), ss, P * sizeof(GSolveState), cudaMemcpyDeviceToHost,
                          st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return FDE_ERR_CUDA;
      bool more = false;
      for (int q = 0; q < P; ++q) {
        const GSolveState& s = ss_host[q];
        if (!s.converged && !s.failed && s.its < hs[q]->p.maxit) more = true;
      }
      if (!more) break;
      if (cudaGraphLaunch(graph[0], st) != cudaSuccess) return FDE_ERR_CUDA;
      launches += graph_launches[0];
    }
    // results out; every problem's solution buffer holds its last iterate
    cudaMemcpyAsync(incycle, ones.data(), P * sizeof(int), cudaMemcpyHostToDevice, st);
    GCHK(launch_g_vec(GV_COPY, copy_out.ent, copy_out.items, copy_out.nitems, all, st));
    if (cudaStreamSynchronize(st) != cudaSuccess) return FDE_ERR_CUDA;
    for (int q = 0; q < P; ++q) {
      const GSolveState& s = ss_host[q];
      fde_stats o{};
      o.iterations = s.its;
      o.restarts = s.restarts;
      o.converged = s.converged;
      o.rel_residual = s.rel_residual;
      o.relaxed = s.relaxed;
      if (stats) stats[q] = o;
      fde_handle* h = hs[q];
      if (s.failed) {
        rc[q] = h->fail(FDE_ERR_NONFINITE, "non-finite value in the grouped solve");
      } else if (!s.converged) {
        rc[q] = h->fail(FDE_ERR_NOT_CONVERGED, "not converged: %d iterations, relative residual %.3e",
                        s.its, s.rel_residual);
      } else {
        rc[q] = FDE_OK;
      }
      if (rc[q] == FDE_OK || rc[q] == FDE_ERR_NOT_CONVERGED) {
        cudaMemcpyAsync(h->u_last, h->hx_out, h->N * 8, cudaMemcpyDeviceToDevice, st);
        h->m++;
      }
    }
    return FDE_OK;
  }
#undef GCHK
};

// C++ entry points used by fde_batch.cu
GroupEngine* group_engine_create(const std::vector<fde_handle*>& hs, cudaStream_t st,
                                 std::string& why) {
  auto* e = new GroupEngine();
  const int r = e->build(hs, st);
  if (r != FDE_OK) {
    why = e->err.empty() ? "grouped engine: allocation failed" : e->err;
    delete e;
    return nullptr;
  }
  return e;
}

void group_engine_destroy(GroupEngine* e) { delete e; }

int group_engine_step(GroupEngine* e, const double* const* u_prev, const double* const* v_half,
                      double* const* u_next, cudaStream_t st, std::vector<int>& rc,
                      fde_stats* stats) {
  return e->step(u_prev, v_half, u_next, st, rc, stats);
}

long long group_engine_launches(const GroupEngine* e) { return e ? e->launches : 0; }

}  // namespace fde
