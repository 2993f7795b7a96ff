// Host side of the per-system batched GMRES (tpp_batch_gmres): validation, the
// work queues of the persistent launches grouped by n, launch shapes, workspace.
// The device code is in k_bgmres.cuh.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "k_bgmres.cuh"

namespace tpp {
namespace bg {
namespace {

constexpr int kWidths[3] = {8, 16, 32};
constexpr size_t kSmemLimit = 227 * 1024;

int width_class(int n) { return n <= 8 ? 0 : (n <= 16 ? 1 : 2); }

struct ClassPlan {
  std::vector<BItem> items;
  int max_nloc = 0, max_n = 0, warps = 8, grid = 0, minb = 1;
  size_t smem = 0, slot_total = 0;
};

struct BatchPlan {
  std::vector<BGroup> groups;
  ClassPlan cls[3];
  size_t off_groups = 0, off_items[3] = {0, 0, 0}, off_ctr = 0, off_stats = 0, off_slots = 0;
  size_t total = 0;
};

const void* kernel_for(int cl, bool mixed, int minb) {
  switch (cl) {
    case 0: return kernel_w8(mixed, minb);
    case 1: return kernel_w16(mixed, minb);
    default: return kernel_w32(mixed, minb);
  }
}

// shared memory of a launch: the lane groups' scratch plus the largest element image
size_t class_smem(const std::vector<BGroup>& G, const std::vector<int>& gids, int NM, int warps,
                  bool mixed) {
  size_t img = 0;
  for (int g : gids) {
    const ElemLayout Li = elem_layout(G[g].dim, G[g].n, true);
    size_t b = al256((size_t)Li.total * (mixed ? 4 : 8));
    if (mixed) b += (size_t)elem_layout(G[g].dim, G[g].n, false).total * 8;
    img = std::max(img, b);
  }
  return (size_t)warps * (32 / NM) * NM * NM * 8 + img;
}

const char* check_opts(const tpp_batch_opts* o) {
  if (!o) return "tpp_batch_opts is NULL";
  if (o->restart < 1 || o->restart > 31) return "restart must be in 1..31";
  if (o->max_iters < 1) return "max_iters must be >= 1";
  if (!(o->rtol > 0.0)) return "rtol must be > 0";
  if (o->prec != TPP_FP64 && o->prec != TPP_FP32) return "prec must be TPP_FP64 or TPP_FP32";
  if (o->prec == TPP_FP32 && (o->max_outer < 1 || !(o->inner_rtol > 0.0 && o->inner_rtol < 1.0)))
    return "mixed precision needs max_outer >= 1 and inner_rtol in (0, 1)";
  for (int k = 0; k < 3; ++k)
    if (o->warps[k] < 0 || o->warps[k] > 8 || o->ctas_per_sm[k] < 0 || o->reg_budget[k] < 0 ||
        o->reg_budget[k] > 2)
      return "warps must be in 0..8, ctas_per_sm >= 0 and reg_budget in 0..2";
  return nullptr;
}

// validate and lay out; b / x may be NULL (sizing only)
std::string plan_batch(tpp_ctx* const* ctxs, int32_t nctx, const double* const* b,
                       double* const* x, const tpp_batch_opts* o, BatchPlan* P) {
  if (const char* why = check_opts(o)) return why;
  if (!ctxs || nctx < 1) return "ctxs must hold nctx >= 1 contexts";
  const bool mixed = o->prec == TPP_FP32;
  std::vector<int> gids[3];
  int dev = -1;
  for (int g = 0; g < nctx; ++g) {
    const tpp_ctx* c = ctxs[g];
    const std::string who = "context " + std::to_string(g) + ": ";
    if (!c) return who + "NULL";
    if (!c->isolated || c->sys_nc > 0)
      return who + "not isolated (every nbr entry must be -1; no coupled system)";
    if (c->mu > c->n || c->curved)
      return who + "over-integrated and curved contexts are not supported";
    if (!two_sided(c)) return who + "needs TPP_FEAT_TWO_SIDED";
    if (c->dim == 2 ? c->n > 32 : c->n > 16) return who + "n above the limit (32 in 2D, 16 in 3D)";
    if (mixed && !(c->features & TPP_FEAT_MIXED)) return who + "mixed precision needs TPP_FEAT_MIXED";
    if (dev >= 0 && c->device != dev) return who + "all contexts must be on one device";
    dev = c->device;
    BGroup G;
    std::memset(&G, 0, sizeof(G));
    G.dim = c->dim;
    G.n = c->n;
    G.R = c->R;
    G.nloc = c->nloc;
    G.E = c->E;
    G.hd = std::pow(c->prob.h, (double)c->dim);
    G.T = c->p<Tables>(c->L.tables);
    G.masks = c->p<uint32_t>(c->L.masks);
    G.d64.cx = c->p<double>(c->L.cx);
    G.d64.cy = c->p<double>(c->L.cy);
    G.d64.cz = (c->dim == 3) ? c->p<double>(c->L.cz) : nullptr;
    G.d64.fa = c->p<double>(c->L.fa);
    G.d64.SA = c->p<double>(c->L.fSA);
    G.d64.SB = c->p<double>(c->L.fSB);
    G.d64.Q1 = c->p<double>(c->L.fQ1);
    G.d64.Q2 = c->p<double>(c->L.fQ2);
    G.d64.T1 = c->p<double>(c->L.fT1);
    G.d64.T2 = c->p<double>(c->L.fT2);
    G.d64.Azi = (c->dim == 3) ? c->p<double>(c->L.fAzi) : nullptr;
    if (mixed) {
      const float* f = c->p<float>(c->L.f32);
      const F32Layout F = f32_layout(c->n, c->E, c->dim, true);
      const float* fo = c->p<float>(c->L.opf);
      const OpF32Layout O = op_f32_layout(c);
      G.d32.cx = fo + O.cx;
      G.d32.cy = fo + O.cy;
      G.d32.cz = (c->dim == 3) ? fo + O.cz : nullptr;
      G.d32.fa = fo + O.fa;
      G.d32.SA = f + F.SA;
      G.d32.SB = f + F.SB;
      G.d32.Q1 = f + F.Q1;
      G.d32.Q2 = f + F.Q2;
      G.d32.T1 = f + F.T1;
      G.d32.T2 = f + F.T2;
      G.d32.Azi = (c->dim == 3) ? f + F.Azi : nullptr;
    }
    if (b || x) {
      if (!c->factors_built) return who + "factors not built";
      if (!b || !x || !b[g] || !x[g]) return who + "b and x must be non-NULL device pointers";
      G.b = b[g];
      G.x = x[g];
    }
    G.iters = o->iters ? o->iters[g] : nullptr;
    G.relres = o->relres ? o->relres[g] : nullptr;
    P->groups.push_back(G);
    gids[width_class(c->n)].push_back(g);
  }
  int cur = -1, sms = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return "no CUDA device";
  if (cur != dev) return "the contexts' device is not the current device";
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return "device query failed";
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += al256(bytes);
    return at;
  };
  P->off_groups = take(P->groups.size() * sizeof(BGroup));
  size_t slots = 0;
  for (int k = 0; k < 3; ++k) {
    ClassPlan& C = P->cls[k];
    if (gids[k].empty()) continue;
    const int NM = kWidths[k];
    // most expensive degree first: per-system work grows like n^(dim+1)
    std::vector<int> order = gids[k];
    std::stable_sort(order.begin(), order.end(), [&](int a, int bb) {
      const BGroup &A = P->groups[a], &B = P->groups[bb];
      return (double)A.nloc * A.n > (double)B.nloc * B.n;
    });
    C.warps = o->warps[k] ? o->warps[k] : 8;
    while (C.warps > 1 && class_smem(P->groups, gids[k], NM, C.warps, mixed) > kSmemLimit)
      --C.warps;
    // items of one system per lane group: an element whose systems converge slowly is
    // spread over many CTAs instead of holding one CTA for all its right-hand sides
    const int ngc = C.warps * (32 / NM);
    for (int g : order) {
      const BGroup& G = P->groups[g];
      C.max_nloc = std::max(C.max_nloc, G.nloc);
      C.max_n = std::max(C.max_n, G.n);
      for (int64_t e = 0; e < G.E; ++e)
        for (int r0 = 0; r0 < G.R; r0 += ngc) C.items.push_back(BItem{g, (int32_t)e, r0, 0});
    }
    C.smem = class_smem(P->groups, gids[k], NM, C.warps, mixed);
    if (C.smem > kSmemLimit) return "an element does not fit in shared memory";
    C.minb = o->reg_budget[k] ? o->reg_budget[k] : (k == 2 ? 1 : 2);
    const void* kern = kernel_for(k, mixed, C.minb);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C.smem) !=
        cudaSuccess)
      return "cudaFuncSetAttribute failed";
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C.warps * 32, C.smem) !=
            cudaSuccess || occ < 1)
      return "no CTA of the batched GMRES fits on an SM";
    const int per_sm = o->ctas_per_sm[k] ? std::min(o->ctas_per_sm[k], occ) : occ;
    C.grid = (int)std::min<int64_t>((int64_t)sms * per_sm, (int64_t)C.items.size());
    const SlotLayout SL = slot_layout(o->restart, C.max_nloc, C.max_n, mixed);
    C.slot_total = (size_t)C.grid * C.warps * (32 / NM) * SL.total;
    slots = std::max(slots, C.slot_total);
    P->off_items[k] = take(C.items.size() * sizeof(BItem));
  }
  P->off_ctr = take(3 * sizeof(int32_t));
  P->off_stats = take(sizeof(BatchStats));
  P->off_slots = take(slots);
  P->total = off;
  return "";
}

}  // namespace
}  // namespace bg
}  // namespace tpp

using namespace tpp;
using namespace tpp::bg;

// six timing events (start / end of each width's launch), destroyed on every return
struct EventSet {
  cudaEvent_t e[6];
  bool ok = true;
  EventSet() {
    for (int k = 0; k < 6; ++k) e[k] = nullptr;
    for (int k = 0; k < 6 && ok; ++k) ok = cudaEventCreate(&e[k]) == cudaSuccess;
  }
  ~EventSet() {
    for (int k = 0; k < 6; ++k)
      if (e[k]) cudaEventDestroy(e[k]);
  }
  cudaEvent_t operator[](int k) const { return e[k]; }
};

#define BG_TRY(call, what)                                 \
  do {                                                     \
    const cudaError_t _e = (call);                         \
    if (_e != cudaSuccess) return cuda_check(_e, what);    \
  } while (0)

extern "C" size_t tpp_batch_workspace_bytes(tpp_ctx* const* ctxs, int32_t nctx,
                                            const tpp_batch_opts* opts) {
  BatchPlan P;
  const std::string why = plan_batch(ctxs, nctx, nullptr, nullptr, opts, &P);
  if (!why.empty()) {
    set_error("tpp_batch_workspace_bytes: " + why);
    return 0;
  }
  return P.total;
}

extern "C" tpp_status tpp_batch_gmres(tpp_ctx* const* ctxs, int32_t nctx, const double* const* b,
                                      double* const* x, const tpp_batch_opts* opts,
                                      tpp_batch_report* report, void* workspace, size_t ws_bytes,
                                      void* stream) {
  if (!report || !workspace || !b || !x) {
    set_error("tpp_batch_gmres: report, workspace, b and x must be non-NULL");
    return TPP_ERR_INVALID_ARG;
  }
  BatchPlan P;
  const std::string why = plan_batch(ctxs, nctx, b, x, opts, &P);
  if (!why.empty()) {
    set_error("tpp_batch_gmres: " + why);
    return TPP_ERR_INVALID_ARG;
  }
  if (ws_bytes < P.total || (reinterpret_cast<uintptr_t>(workspace) & 255u)) {
    set_error("tpp_batch_gmres: workspace smaller than tpp_batch_workspace_bytes or not "
              "256-byte aligned");
    return TPP_ERR_WORKSPACE;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  const bool mixed = opts->prec == TPP_FP32;
  BG_TRY(cudaMemcpyAsync(ws + P.off_groups, P.groups.data(), P.groups.size() * sizeof(BGroup),
                         cudaMemcpyHostToDevice, s),
         "copy groups");
  for (int k = 0; k < 3; ++k)
    if (!P.cls[k].items.empty())
      BG_TRY(cudaMemcpyAsync(ws + P.off_items[k], P.cls[k].items.data(),
                             P.cls[k].items.size() * sizeof(BItem), cudaMemcpyHostToDevice, s),
             "copy items");
  BG_TRY(cudaMemsetAsync(ws + P.off_ctr, 0, 3 * sizeof(int32_t), s), "memset");
  BG_TRY(cudaMemsetAsync(ws + P.off_stats, 0, sizeof(BatchStats), s), "memset");
  BParams bp;
  std::memset(&bp, 0, sizeof(bp));
  bp.groups = reinterpret_cast<const BGroup*>(ws + P.off_groups);
  bp.m = opts->restart;
  bp.max_iters = opts->max_iters;
  bp.max_outer = mixed ? opts->max_outer : 1;
  bp.mixed = mixed ? 1 : 0;
  bp.rtol = opts->rtol;
  bp.inner_rtol = mixed ? opts->inner_rtol : opts->rtol;
  bp.slots = ws + P.off_slots;
  bp.st = reinterpret_cast<BatchStats*>(ws + P.off_stats);
  EventSet ev;
  if (!ev.ok) return cuda_check(cudaErrorMemoryAllocation, "cudaEventCreate");
  int launches = 0;
  int64_t systems = 0;
  for (const BGroup& G : P.groups) systems += G.E * G.R;
  for (int k = 2; k >= 0; --k) {            // widest (most expensive) class first
    const ClassPlan& C = P.cls[k];
    if (C.items.empty()) continue;
    bp.items = reinterpret_cast<const BItem*>(ws + P.off_items[k]);
    bp.nitems = (int32_t)C.items.size();
    bp.counter = reinterpret_cast<int32_t*>(ws + P.off_ctr) + k;
    ClassArgs ca{C.max_nloc, C.max_n};
    void* args[] = {&bp, &ca};
    BG_TRY(cudaEventRecord(ev[2 * k], s), "event");
    BG_TRY(cudaLaunchKernel(kernel_for(k, mixed, C.minb), dim3(C.grid), dim3(C.warps * 32), args,
                            C.smem, s),
           "k_bgmres");
    BG_TRY(cudaEventRecord(ev[2 * k + 1], s), "event");
    count_launch();
    ++launches;
  }
  BatchStats st;
  BG_TRY(cudaMemcpyAsync(&st, ws + P.off_stats, sizeof(st), cudaMemcpyDeviceToHost, s),
         "read stats");
  BG_TRY(cudaStreamSynchronize(s), "tpp_batch_gmres sync");
  std::memset(report, 0, sizeof(*report));
  report->systems = systems;
  report->total_iters = (int64_t)st.total_iters;
  report->max_iters = st.max_iters;
  report->unconverged = st.unconverged;
  report->max_outer = st.outer_max;
  report->launches = launches;
  report->max_relres = st.max_relres;
  for (int k = 0; k < 3; ++k) {
    float ms = 0.0f;
    if (!P.cls[k].items.empty() && cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]) == cudaSuccess)
      report->launch_ms[k] = ms;
  }
  if (st.unconverged > 0) {
    set_error("tpp_batch_gmres: " + std::to_string(st.unconverged) +
              " system(s) above rtol at exit");
    return TPP_ERR_NOT_CONVERGED;
  }
  return TPP_OK;
}
