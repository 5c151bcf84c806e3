// cfr_api.cu — the C ABI of libcfr.so (declared in include/cfr.h): arena
// planning and binding, the three execution forms (per-level launches, one
// replayed CUDA graph per iteration, one persistent kernel per call), the
// FP64 exact best response, and state read-out in the caller's slot order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/cfr.h"
#include "compiled.h"
#include "launch.h"

using namespace cfr;

static thread_local std::string g_err;

static int set_err(int code, const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return set_err(CFR_ERR_DEVICE, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                     __FILE__, __LINE__);                                                          \
  } while (0)

extern "C" const char *cfr_last_error(void) { return g_err.c_str(); }

struct Buf {
  size_t off = 0, bytes = 0;
};

// Largest lane group at depths whose sets are tiled (member order).
constexpr int kTiledLanes = 32 / kTileSets;

struct cfr_handle {
  Compiled c;
  cfr_options opt{};
  int precision = CFR_P32, exec_form = CFR_EXEC_GRAPH, rule = 0, order = 0;
  int maxa_tier = 8;           // 4, 8 or 64: register arrays of the per-set code
  std::vector<int> level_lanes;  // lanes per information set, per depth
  std::vector<int> pull_grid;    // member order: blocks of the forward launch of depth d (set at bind; 0 = none)
  int persist_lanes = 8;
  std::vector<LevelWork> levels;
  // arena layout
  Buf b_iset_slot, b_iset_mem, b_iset_vb, b_mem_vs, b_ch_vb, b_ch_nch, b_ch_vs, b_spec_slot, b_levels;
  Buf b_wide_vb, b_wide_nch, b_wide_vs, b_wide_chunk, b_wide_part, b_wide_cnt;
  Buf b_int_slot, b_int_mask, b_int_cirank, b_big_irank, b_int_edge, b_iset_rank, b_mem_irank, b_wide_irank;
  Buf b_reach, b_v, b_sigma, b_R, b_avg, b_tmpl, b_sbs, b_reach2, b_vb, b_vavg, b_t, b_bar, b_err, b_out;
  // streaming backward (FP32, member order): set descriptors, chunks, and per
  // depth the chunk range (stream_c0[d] .. stream_c0[d+1]) and whether the
  // depth can stream (every group fits one stage)
  std::vector<SetInfo> set_info;
  std::vector<StreamChunk> stream_chunks;
  std::vector<int32_t> stream_c0, stream_ok;
  Buf b_set_info, b_stream_chunks;
  size_t plan_bytes = 0;
  char *arena = nullptr;
  bool bound = false;
  std::vector<void *> pinned;  // host ranges page-locked by cfr_pin_host
  // graph form: one iteration per graph (gexec) and, with graph_iters = k > 1,
  // k iterations per graph (gexec_k)
  cudaGraphExec_t gexec = nullptr;
  cudaGraphExec_t gexec_k = nullptr;
  int64_t graph_kernels = 0, graph_k_kernels = 0;  // kernel nodes of the captured graphs
  cudaStream_t cap_stream = nullptr;
  // persistent form
  int persist_grid = 0;
  int test_missing_arrivals = 0;  // fault-injection hook: barriers wait for blocks that never come
  int test_fail_capture = 0;      // test hook: treat the next graph capture as failed
  bool capture_warned = false;    // the capture-failure warning is printed once per handle
  int64_t iteration_host = 0;  // iterations enqueued since bind/reset (bookkeeping)
  template <typename X> X *p(const Buf &b) const { return reinterpret_cast<X *>(arena + b.off); }
};

static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

static void drop_graphs(cfr_handle *h);

static void plan(cfr_handle *h) {
  const Compiled &c = h->c;
  const size_t T = h->precision == CFR_P64 ? 8 : 4;
  size_t cur = 0;
  auto take = [&](Buf &b, size_t bytes) {
    b.off = cur;
    b.bytes = bytes;
    cur = align_up(cur + std::max<size_t>(bytes, 1));
  };
  const size_t n_narrow = c.ch_vb.size();
  take(h->b_iset_slot, 4 * (c.I + 1));
  take(h->b_iset_mem, 4 * (c.I + 1));
  take(h->b_iset_vb, 4 * c.I);
  take(h->b_mem_vs, 4 * c.n_dec);
  take(h->b_ch_vb, 4 * n_narrow);
  take(h->b_ch_nch, 4 * n_narrow);
  take(h->b_ch_vs, 4 * n_narrow);
  take(h->b_spec_slot, 4 * c.A);
  take(h->b_levels, sizeof(LevelWork) * std::max<int64_t>(c.D, 1));
  take(h->b_wide_vb, 4 * c.n_wide);
  take(h->b_wide_nch, 4 * c.n_wide);
  take(h->b_wide_vs, 4 * c.n_wide);
  take(h->b_wide_chunk, 4 * (c.n_wide + 1));
  take(h->b_wide_part, 3 * 8 * (size_t)c.wide_chunk.back());
  take(h->b_wide_cnt, 4 * c.n_wide);
  // push records (breadth-first or value-slot order) or pull edges (member order)
  take(h->b_int_slot, 4 * c.int_slot.size());
  take(h->b_int_mask, 4 * c.int_mask.size());
  take(h->b_int_cirank, 4 * c.int_cirank.size());
  take(h->b_big_irank, 4 * c.big_irank.size());
  take(h->b_int_edge, 4 * c.int_edge.size());
  take(h->b_iset_rank, 4 * c.iset_rank.size());
  take(h->b_mem_irank, c.int_edge.empty() ? 4 * c.n_dec : 0);  // member order: ranks follow from k
  take(h->b_wide_irank, 4 * c.wide_irank.size());
  take(h->b_reach, 2 * T * std::max<int64_t>(c.n_int, 1));  // internal nodes only
  take(h->b_v, T * c.N);  // value slots
  take(h->b_sigma, T * (c.A + 1));
  take(h->b_R, 8 * c.A);
  take(h->b_avg, 8 * c.A);
  take(h->b_tmpl, 8 * c.N);  // template in slot order
  take(h->b_sbs, 8 * c.A);
  take(h->b_reach2, 16 * std::max<int64_t>(c.n_int, 1));
  take(h->b_vb, 16 * c.N);
  take(h->b_vavg, 8 * c.N);
  take(h->b_t, 8);
  take(h->b_bar, 16);
  take(h->b_err, 16);
  take(h->b_out, 8 * std::max<int64_t>(c.A, 2) + 64);
  take(h->b_set_info, sizeof(SetInfo) * h->set_info.size());
  take(h->b_stream_chunks, sizeof(StreamChunk) * h->stream_chunks.size());
  h->plan_bytes = cur;
}

// Set descriptors and chunks of the streaming backward (FP32, member order,
// sets of at most 8 actions). A group is a tile of kTileSets sets (members'
// reach interleaved) or one untiled set; a chunk is a run of whole groups of
// one depth whose staged bytes (stream_layout) fit one stage. A depth whose
// largest group does not fit cannot stream.
static void build_stream(cfr_handle *h) {
  const Compiled &c = h->c;
  h->set_info.clear();
  h->stream_chunks.clear();
  h->stream_c0.assign(c.D + 1, 0);
  h->stream_ok.assign(c.D, 0);
  if (h->precision != CFR_P32 || c.int_edge.empty() || c.max_act > 8 || c.I == 0) return;
  h->set_info.resize(c.I);
  for (int64_t d = 0; d < c.D; ++d) {
    const int32_t p2 = c.level_iset[2 * d + 1];
    for (int32_t I = c.level_iset[2 * d]; I < c.level_iset[2 * d + 2];) {
      const bool tile = c.iset_rank[2 * I + 1] == kTileSets;
      const int32_t G = tile ? kTileSets : 1;
      for (int32_t j = 0; j < G; ++j) {
        SetInfo &si = h->set_info[I + j];
        si.sb = c.iset_slot[I + j];
        si.na = c.iset_slot[I + j + 1] - si.sb;
        si.m0 = c.iset_mem[I + j];
        si.nm = c.iset_mem[I + j + 1] - si.m0;
        si.vb = c.iset_vb[I + j];
        si.rank0 = c.iset_rank[2 * (I + j)];
        si.rstep = c.iset_rank[2 * (I + j) + 1];
        si.flags = (j == 0 ? G : 0) | ((I + j) >= p2 ? 1 << 8 : 0);
      }
      I += G;
    }
  }
  auto make = [&](int32_t I0, int32_t I1) {
    StreamChunk k{};
    int64_t rlo = INT64_MAX, rhi = 0, vlo = INT64_MAX, vhi = 0, mlo = INT64_MAX, mhi = 0, slo = INT64_MAX, shi = 0;
    for (int32_t I = I0; I < I1; ++I) {
      const SetInfo &si = h->set_info[I];
      rlo = std::min<int64_t>(rlo, si.rank0);
      rhi = std::max<int64_t>(rhi, (int64_t)si.rank0 + (int64_t)(si.nm - 1) * si.rstep + 1);
      vlo = std::min<int64_t>(vlo, si.vb);
      vhi = std::max<int64_t>(vhi, (int64_t)si.vb + (int64_t)si.nm * si.na);
      mlo = std::min<int64_t>(mlo, si.m0);
      mhi = std::max<int64_t>(mhi, (int64_t)si.m0 + si.nm);
      slo = std::min<int64_t>(slo, si.sb);
      shi = std::max<int64_t>(shi, (int64_t)si.sb + si.na);
    }
    k.I0 = I0;
    k.I1 = I1;
    k.ra = (int32_t)(rlo & ~int64_t(1));
    k.nra = (int32_t)(((rhi + 1) & ~int64_t(1)) - k.ra);
    k.va = (int32_t)(vlo & ~int64_t(3));
    k.nva = (int32_t)(((vhi + 3) & ~int64_t(3)) - k.va);
    k.ka = (int32_t)(mlo & ~int64_t(3));
    k.nka = (int32_t)(((mhi + 3) & ~int64_t(3)) - k.ka);
    k.sa = (int32_t)(slo & ~int64_t(3));
    k.nsa = (int32_t)(((shi + 3) & ~int64_t(3)) - k.sa);
    return k;
  };
  // chance nodes [i0, i1) of one depth: their children's value slots
  // [first child of i0, end of i1 - 1's) and their chance-array entries,
  // widened to 16-byte boundaries
  auto make_chance = [&](int32_t i0, int32_t i1) {
    StreamChunk k{};
    k.kind = kChunkChance;
    k.I0 = i0;
    k.I1 = i1;
    const int64_t lo = c.ch_vb[i0], hi = (int64_t)c.ch_vb[i1 - 1] + c.ch_nch[i1 - 1];
    k.va = (int32_t)(lo & ~int64_t(3));
    k.nva = (int32_t)(std::max<int64_t>(((hi + 3) & ~int64_t(3)) - k.va, 4));
    k.ka = i0 & ~3;
    k.nka = ((i1 + 3) & ~3) - k.ka;
    return k;
  };
  for (int64_t d = 0; d < c.D; ++d) {
    h->stream_c0[d] = (int32_t)h->stream_chunks.size();
    const int32_t is0 = c.level_iset[2 * d], is1 = c.level_iset[2 * d + 2];
    // depth 0 holds only the root (and advances t); wide chance nodes are
    // summed by the per-level kernel's chunk blocks, which the streaming
    // kernel does not have
    bool ok = d > 0 && is1 > is0 && c.level_wide[d + 1] == c.level_wide[d];
    std::vector<StreamChunk> ch;
    for (int32_t I = is0; ok && I < is1;) {
      int32_t J = I + (h->set_info[I].flags & 7);
      if (!stream_fits(stream_layout(make(I, J)))) { ok = false; break; }
      while (J < is1) {  // extend by whole groups while the stage holds them
        const int32_t K = J + (h->set_info[J].flags & 7);
        if (!stream_fits(stream_layout(make(I, K)))) break;
        J = K;
      }
      ch.push_back(make(I, J));
      I = J;
    }
    // then the depth's narrow chance nodes, in chunks of consecutive nodes
    // whose children (consecutive value slots) and chance-array entries fit
    // a stage; each node's child run must lie inside its chunk's
    const int32_t q0 = c.level_chance[d], q1 = c.level_chance[d + 1];
    for (int32_t i = q0; ok && i < q1;) {
      int32_t j = i + 1;
      if (!chance_fits(make_chance(i, j))) { ok = false; break; }
      while (j < q1 && j - i < kStreamChanceMax && chance_fits(make_chance(i, j + 1))) ++j;
      const StreamChunk k = make_chance(i, j);
      for (int32_t q = i; q < j; ++q)
        if (c.ch_vb[q] < k.va || (int64_t)c.ch_vb[q] + c.ch_nch[q] > (int64_t)k.va + k.nva) ok = false;
      ch.push_back(k);
      i = j;
    }
    if (ok) {
      h->stream_ok[d] = 1;
      h->stream_chunks.insert(h->stream_chunks.end(), ch.begin(), ch.end());
    }
  }
  h->stream_c0[c.D] = (int32_t)h->stream_chunks.size();
}

// --------------------------------------------------------------- compile
extern "C" int cfr_compile(const cfr_game_spec *spec, const cfr_options *opt, cfr_handle **out) {
  if (!spec || !out) return set_err(CFR_ERR_ARG, "cfr_compile: null argument");
  *out = nullptr;
  cfr_handle *h = new (std::nothrow) cfr_handle();
  if (!h) return set_err(CFR_ERR_HOST_MEMORY, "cfr_compile: out of host memory");
  if (opt) h->opt = *opt;
  else { h->opt.precision = CFR_P32; h->opt.exec_form = CFR_EXEC_AUTO; }
  if (h->opt.precision != CFR_P64 && h->opt.precision != CFR_P32) { delete h; return set_err(CFR_ERR_ARG, "bad precision"); }
  if (h->opt.exec_form < 0 || h->opt.exec_form > 3) { delete h; return set_err(CFR_ERR_ARG, "bad exec_form"); }
  if (h->opt.rule != CFR_RULE_CFR_PLUS && h->opt.rule != CFR_RULE_CFR && h->opt.rule != CFR_RULE_PCFR_PLUS) { delete h; return set_err(CFR_ERR_ARG, "bad rule"); }
  if (h->opt.order != CFR_ORDER_SIMULTANEOUS && h->opt.order != CFR_ORDER_ALTERNATING) { delete h; return set_err(CFR_ERR_ARG, "bad order"); }
  const int lp = h->opt.lanes_per_set;
  if (lp != 0 && lp != 1 && lp != 2 && lp != 4 && lp != 8 && lp != 16 && lp != 32 && lp != kThreads && lp != kStreamLanes) { delete h; return set_err(CFR_ERR_ARG, "lanes_per_set must be 0, 1, 2, 4, 8, 16, 32, 256 or 512"); }
  if (lp == kStreamLanes && (h->opt.precision != CFR_P32 || h->opt.reach_order != CFR_REACH_MEMBERS)) { delete h; return set_err(CFR_ERR_ARG, "lanes_per_set 512 (streaming) needs CFR_P32 and CFR_REACH_MEMBERS"); }
  std::string err;
  if (h->opt.reach_order < CFR_REACH_MEMBERS || h->opt.reach_order > CFR_REACH_SLOTS) { delete h; return set_err(CFR_ERR_ARG, "bad reach_order"); }
  if (h->opt.member_tiles < CFR_TILES_AUTO || h->opt.member_tiles > CFR_TILES_ON) { delete h; return set_err(CFR_ERR_ARG, "bad member_tiles"); }
  if (h->opt.launch_overlap != CFR_OVERLAP_AUTO && h->opt.launch_overlap != CFR_OVERLAP_ON &&
      h->opt.launch_overlap != CFR_OVERLAP_OFF) { delete h; return set_err(CFR_ERR_ARG, "bad launch_overlap"); }
  if (h->opt.graph_iters < 0 || h->opt.graph_iters > 1000) { delete h; return set_err(CFR_ERR_ARG, "graph_iters must be in [0, 1000]"); }
  int rc = compile_game(*spec, h->c, err, h->opt.reach_order, h->opt.member_tiles);
  if (rc != CFR_OK) { delete h; return set_err(rc, "cfr_compile: %s", err.c_str()); }
  const Compiled &c = h->c;
  if (lp != 0 && (lp < 4 || lp == kThreads || lp == kStreamLanes) && c.max_act > 8) { delete h; return set_err(CFR_ERR_ARG, "lanes_per_set 1, 2, 256 or 512 needs sets of at most 8 actions"); }
  h->precision = h->opt.precision;
  h->rule = h->opt.rule;
  h->order = h->opt.order;
  h->maxa_tier = c.max_act <= 4 ? 4 : (c.max_act <= 8 ? 8 : 64);
  h->exec_form = h->opt.exec_form;
  // AUTO: the persistent kernel only where it was measured faster than graph
  // replay per iteration (one GB300: P32 up to about 400 nodes, graph from
  // about 1,200; P64 up to about 300, graph from about 400)
  if (h->exec_form == CFR_EXEC_AUTO)
    h->exec_form = c.N <= (h->opt.precision == CFR_P32 ? 768 : 350) ? CFR_EXEC_PERSISTENT : CFR_EXEC_GRAPH;
  // lanes per information set: the smallest group that covers the mean set
  auto pick = [](double mean) { return mean <= 4.0 ? 4 : mean <= 8.0 ? 8 : mean <= 16.0 ? 16 : 32; };
  // (tiled depths: at most one tile of sets per warp's worth of lanes, so a
  // warp's member reads stay one run)
  h->level_lanes.assign(c.D, 8);
  h->pull_grid.assign(c.D, 0);
  double tot_mem = 0.0;
  bool any_tiled = false;
  build_stream(h);
  for (int64_t d = 0; d < c.D; ++d) {
    h->level_lanes[d] = (lp && lp != kStreamLanes) ? lp : pick(c.level_mean_members[d]);
    if (lp == kStreamLanes && h->stream_ok[d]) h->level_lanes[d] = kStreamLanes;
    if ((!lp || (lp == kStreamLanes && !h->stream_ok[d])) && c.level_tiled[d])
      h->level_lanes[d] = std::min(h->level_lanes[d], kTiledLanes);
    any_tiled = any_tiled || c.level_tiled[d];
    tot_mem += c.level_mean_members[d] * (c.level_iset[2 * d + 2] - c.level_iset[2 * d]);
  }
  // the persistent kernel runs lane groups of at most a warp
  h->persist_lanes = lp ? std::min(lp, 32) : pick(c.I > 0 ? tot_mem / (double)c.I : 1.0);
  if (!lp && any_tiled) h->persist_lanes = std::min(h->persist_lanes, kTiledLanes);
  h->levels.resize(c.D);
  for (int64_t d = 0; d < c.D; ++d) {
    LevelWork &w = h->levels[d];
    w.ib = c.level_int[d];
    w.ie = c.level_int[d + 1];
    w.lb = c.level_begin[d];
    w.le = c.level_begin[d + 1];
    w.ch0 = c.level_chance[d];
    w.ch1 = c.level_chance[d + 1];
    w.is0 = c.level_iset[2 * d];
    w.is2 = c.level_iset[2 * d + 1];
    w.is1 = c.level_iset[2 * d + 2];
    w.wd0 = c.level_wide[d];
    w.wd1 = c.level_wide[d + 1];
    w.wc0 = c.wide_chunk[w.wd0];
    w.wc1 = c.wide_chunk[w.wd1];
    w.fan = 0;  // a chance node of this depth has its children written warp-wide
    for (int64_t q = c.level_int[d]; q < c.level_int[d + 1] && !w.fan && !c.int_mask.empty(); ++q) {
      const uint32_t m = c.int_mask[q];
      if (c.int_slot[q] < 0 && m != 0u && ((m & kBigNode) || __builtin_popcount(m) > kFanLight)) w.fan = 1;
    }
  }
  plan(h);
  *out = h;
  return CFR_OK;
}

extern "C" void cfr_destroy(cfr_handle *h) {
  if (!h) return;
  for (void *p : h->pinned) cudaHostUnregister(p);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->gexec_k) cudaGraphExecDestroy(h->gexec_k);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

extern "C" int cfr_get_counts(const cfr_handle *h, cfr_counts *o) {
  if (!h || !o) return set_err(CFR_ERR_ARG, "cfr_get_counts: null argument");
  const Compiled &c = h->c;
  o->n_nodes = c.N; o->n_edges = c.E; o->n_infosets = c.I; o->n_slots = c.A;
  o->n_internal = c.n_int; o->n_decision = c.n_dec; o->n_chance = c.n_chance; o->n_terminal = c.n_term;
  o->depth_blocks = c.D; o->max_actions = c.max_act;
  o->algo_bytes_per_iter = algo_bytes_per_iter(c, h->precision) * (h->order == CFR_ORDER_ALTERNATING ? 2 : 1);
  o->upload_bytes = (int64_t)(h->b_iset_slot.bytes + h->b_iset_mem.bytes + h->b_iset_vb.bytes + h->b_mem_vs.bytes +
                              h->b_ch_vb.bytes + h->b_ch_nch.bytes + h->b_ch_vs.bytes + h->b_spec_slot.bytes + h->b_levels.bytes +
                              h->b_wide_vb.bytes + h->b_wide_nch.bytes + h->b_wide_vs.bytes +
                              h->b_wide_chunk.bytes + h->b_tmpl.bytes + h->b_int_slot.bytes +
                              h->b_int_mask.bytes + h->b_int_cirank.bytes + h->b_big_irank.bytes + h->b_int_edge.bytes + h->b_iset_rank.bytes +
                              h->b_mem_irank.bytes + h->b_wide_irank.bytes + h->b_set_info.bytes +
                              h->b_stream_chunks.bytes);
  o->iteration = h->iteration_host;
  o->exec_form = h->exec_form;
  o->graph_kernels = h->gexec ? h->graph_kernels : 0;
  o->graph_k_kernels = h->gexec_k ? h->graph_k_kernels : 0;
  o->lanes_per_set = h->exec_form == CFR_EXEC_PERSISTENT ? h->persist_lanes : (c.D > 0 ? h->level_lanes[c.D - 1] : 0);
  return CFR_OK;
}

extern "C" int cfr_plan(const cfr_handle *h, size_t *bytes) {
  if (!h || !bytes) return set_err(CFR_ERR_ARG, "cfr_plan: null argument");
  *bytes = h->plan_bytes;
  return CFR_OK;
}

static GameView game_view(const cfr_handle *h) {
  GameView g;
  g.iset_slot = h->p<int32_t>(h->b_iset_slot);
  g.iset_mem = h->p<int32_t>(h->b_iset_mem);
  g.iset_vb = h->p<int32_t>(h->b_iset_vb);
  g.mem_vs = h->p<int32_t>(h->b_mem_vs);
  g.ch_vb = h->p<int32_t>(h->b_ch_vb);
  g.ch_nch = h->p<int32_t>(h->b_ch_nch);
  g.ch_vs = h->p<int32_t>(h->b_ch_vs);
  g.wide_vb = h->p<int32_t>(h->b_wide_vb);
  g.wide_nch = h->p<int32_t>(h->b_wide_nch);
  g.wide_vs = h->p<int32_t>(h->b_wide_vs);
  g.wide_chunk = h->p<int32_t>(h->b_wide_chunk);
  g.wide_part = h->p<double>(h->b_wide_part);
  g.wide_cnt = h->p<unsigned>(h->b_wide_cnt);
  g.int_slot = h->p<int32_t>(h->b_int_slot);
  g.int_mask = h->p<uint32_t>(h->b_int_mask);
  g.int_cirank = h->p<int32_t>(h->b_int_cirank);
  g.big_irank = h->p<int32_t>(h->b_big_irank);
  g.int_edge = h->c.int_edge.empty() ? nullptr : h->p<int2>(h->b_int_edge);
  g.iset_rank = h->c.iset_rank.empty() ? nullptr : h->p<int2>(h->b_iset_rank);
  g.mem_irank = h->c.int_edge.empty() ? h->p<int32_t>(h->b_mem_irank) : nullptr;
  g.wide_irank = h->p<int32_t>(h->b_wide_irank);
  return g;
}

template <typename T> static StateView<T> state_view(const cfr_handle *h) {
  StateView<T> s;
  s.reach = h->p<vec2_t<T>>(h->b_reach);
  s.v = h->p<T>(h->b_v);
  s.sigma = h->p<T>(h->b_sigma);
  s.R = h->p<double>(h->b_R);
  s.avg = h->p<double>(h->b_avg);
  s.t = h->p<long long>(h->b_t);
  return s;
}

static int grid_for(int64_t work, int per_block) {
  int64_t b = (work + per_block - 1) / per_block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

static int device_sms() {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      nsm = 148;
  }
  return nsm;
}

// Blocks of the pulling forward launch of depth d (member order): at most
// enough for its nodes, kPull per thread.
static int pull_need(const cfr_handle *h, int64_t d) {
  const LevelWork &n = h->levels[d + 1];
  return grid_for((n.ie - n.ib + kPull - 1) / kPull, kThreads);
}

// The grid of every pulling forward launch: the blocks the SMs hold at
// once (one wave), so that the grid-stride loop walks the nodes in rounds of
// consecutive ranks and the parents a round gathers are still in L2 when the
// next round's neighbours read them (two waves split every round's range
// between the waves). Smaller grids run some depths faster alone but slow
// the iteration down inside the graph, so the autotuner leaves this alone.
template <typename T>
static int default_pull_grids(cfr_handle *h) {
  const Compiled &c = h->c;
  if (c.int_edge.empty()) return CFR_OK;
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fwd_pull_kernel<T>, kThreads, 0));
  for (int64_t d = 0; d + 1 < c.D; ++d) h->pull_grid[d] = std::min(pull_need(h, d), std::max(occ, 1) * device_sms());
  return CFR_OK;
}

// Forward launch of depth d. Member order: the internal nodes of depth d + 1
// pull their reach (no launch for the deepest depth). Breadth-first and
// value-slot orders: nb blocks over depth d's internal nodes push to their
// children, then one block per wide chunk; depths with many-child chance
// nodes take the form that writes those children warp-wide.
template <typename T>
static int launch_fwd(const cfr_handle *h, int64_t d, cudaStream_t s, const GameView &g, const T *sigma,
                      vec2_t<T> *reach, bool pdl = false) {
  const LevelWork &w = h->levels[d];
  if (g.int_edge) {  // member order: the next depth's internal nodes pull their reach
    if (d + 1 >= h->c.D) return CFR_OK;
    const LevelWork &n = h->levels[d + 1];
    const int nb = h->pull_grid[d] > 0 ? h->pull_grid[d] : pull_need(h, d);
    CK(launch_k(fwd_pull_kernel<T>, nb, kThreads, 0, s, pdl, g, sigma, reach, n.ib, n.ie));
    return CFR_OK;
  }
  const int nb = grid_for((w.ie - w.ib + 3) / 4, kThreads);
  if (w.fan) CK(launch_k(fwd_level_kernel<T, true>, nb + (w.wc1 - w.wc0), kThreads, 0, s, pdl, g, sigma, reach, w, nb));
  else CK(launch_k(fwd_level_kernel<T, false>, nb + (w.wc1 - w.wc0), kThreads, 0, s, pdl, g, sigma, reach, w, nb));
  return CFR_OK;
}

template <typename T>
static int init_state(cfr_handle *h, cudaStream_t s) {
  const Compiled &c = h->c;
  init_state_kernel<T><<<grid_for(std::max(c.A, c.I), kThreads), kThreads, 0, s>>>(
      h->p<int32_t>(h->b_iset_slot), (int32_t)c.I, h->p<T>(h->b_sigma), h->p<double>(h->b_R),
      h->p<double>(h->b_avg), (int32_t)c.A, h->p<long long>(h->b_t), h->p<vec2_t<T>>(h->b_reach),
      h->p<double2>(h->b_reach2));
  CK(cudaGetLastError());
  h->iteration_host = 0;
  return CFR_OK;
}

template <typename T>
static int init_values(cfr_handle *h, cudaStream_t s) {
  const Compiled &c = h->c;
  CK(cudaMemcpyAsync(h->p<double>(h->b_tmpl), c.tmpl_vs.data(), 8 * c.N, cudaMemcpyHostToDevice, s));
  init_values_kernel<T><<<grid_for(c.N, kThreads), kThreads, 0, s>>>(
      h->p<double>(h->b_tmpl), (int32_t)c.N, h->p<T>(h->b_v), h->p<double2>(h->b_vb), h->p<double>(h->b_vavg));
  CK(cudaGetLastError());
  return CFR_OK;
}

// The host ranges cfr_bind copies from, and the value template.
static std::vector<std::pair<const void *, size_t>> host_ranges(const cfr_handle *h) {
  const Compiled &c = h->c;
  std::vector<std::pair<const void *, size_t>> r = {
      {c.iset_slot.data(), 4 * c.iset_slot.size()},   {c.iset_mem.data(), 4 * c.iset_mem.size()},
      {c.iset_vb.data(), 4 * c.iset_vb.size()},       {c.mem_vs.data(), 4 * c.mem_vs.size()},
      {c.ch_vb.data(), 4 * c.ch_vb.size()},           {c.ch_nch.data(), 4 * c.ch_nch.size()},
      {c.ch_vs.data(), 4 * c.ch_vs.size()},           {c.spec_slot_of.data(), 4 * c.spec_slot_of.size()},
      {c.wide_vb.data(), 4 * c.wide_vb.size()},       {c.wide_nch.data(), 4 * c.wide_nch.size()},
      {c.wide_vs.data(), 4 * c.wide_vs.size()},       {c.wide_chunk.data(), 4 * c.wide_chunk.size()},
      {c.int_slot.data(), 4 * c.int_slot.size()},     {c.int_mask.data(), 4 * c.int_mask.size()},
      {c.int_cirank.data(), 4 * c.int_cirank.size()}, {c.big_irank.data(), 4 * c.big_irank.size()},
      {c.int_edge.data(), 4 * c.int_edge.size()},     {c.iset_rank.data(), 4 * c.iset_rank.size()},
      {c.mem_irank.data(), 4 * c.mem_irank.size()},   {c.wide_irank.data(), 4 * c.wide_irank.size()},
      {c.tmpl_vs.data(), 8 * c.tmpl_vs.size()},
      {h->set_info.data(), sizeof(SetInfo) * h->set_info.size()},
      {h->stream_chunks.data(), sizeof(StreamChunk) * h->stream_chunks.size()}};
  return r;
}

extern "C" int cfr_set_chance_sums(const cfr_handle *h, const double *root_w, double *mass, double *wsum) {
  if (!h || (!mass && h->c.I > 0) || (root_w && !wsum && h->c.I > 0))
    return set_err(CFR_ERR_ARG, "cfr_set_chance_sums: null argument");
  const Compiled &c = h->c;
  std::vector<int32_t> owner;  // root outcome above each node (breadth-first ids: parents first)
  if (root_w) {
    if (c.N == 0 || c.child_begin[1] == c.child_begin[0] || c.node_slot[0] >= 0)
      return set_err(CFR_ERR_UNSUPPORTED, "cfr_set_chance_sums: the root is not a chance node");
    owner.assign(c.N, -1);
    for (int32_t x = c.child_begin[0]; x < c.child_begin[1]; ++x) owner[x] = x - c.child_begin[0];
    for (int64_t h2 = 1; h2 < c.N; ++h2)
      for (int32_t x = c.child_begin[h2]; x < c.child_begin[h2 + 1]; ++x) owner[x] = owner[h2];
  }
  for (int64_t q = 0; q < c.I; ++q) {
    double m = 0.0, w = 0.0;
    for (int32_t k = c.iset_mem[q]; k < c.iset_mem[q + 1]; ++k) {
      const int32_t hh = c.mem_node[k];
      m += c.pc[hh];
      if (root_w) w += c.pc[hh] * root_w[owner[hh]];
    }
    const int32_t sp = c.spec_set_of[q];
    mass[sp] = m;
    if (root_w) wsum[sp] = w;
  }
  return CFR_OK;
}

extern "C" int cfr_pin_host(cfr_handle *h, int pin) {
  if (!h) return set_err(CFR_ERR_ARG, "cfr_pin_host: null handle");
  if (!pin) {
    for (void *p : h->pinned) cudaHostUnregister(p);
    h->pinned.clear();
    return CFR_OK;
  }
  if (!h->pinned.empty()) return CFR_OK;
  for (const auto &r : host_ranges(h)) {
    if (r.second == 0) continue;
    void *p = const_cast<void *>(r.first);
    const cudaError_t e = cudaHostRegister(p, r.second, cudaHostRegisterDefault);
    if (e == cudaErrorHostMemoryAlreadyRegistered) {
      cudaGetLastError();  // a page shared with a range pinned before: leave it
      continue;
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      for (void *q : h->pinned) cudaHostUnregister(q);
      h->pinned.clear();
      return set_err(CFR_ERR_DEVICE, "cfr_pin_host: %s", cudaGetErrorString(e));
    }
    h->pinned.push_back(p);
  }
  return CFR_OK;
}

extern "C" int cfr_bind(cfr_handle *h, void *arena, size_t bytes, void *stream) {
  if (!h || !arena) return set_err(CFR_ERR_ARG, "cfr_bind: null argument");
  if (bytes < h->plan_bytes) return set_err(CFR_ERR_ARENA_SMALL, "cfr_bind: arena has %zu bytes, plan needs %zu", bytes, h->plan_bytes);
  if (reinterpret_cast<uintptr_t>(arena) % 256 != 0) return set_err(CFR_ERR_ARG, "cfr_bind: arena must be 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  drop_graphs(h);
  h->arena = (char *)arena;
  const Compiled &c = h->c;
  auto up = [&](const Buf &b, const void *src, size_t n) -> int {
    if (n) CK(cudaMemcpyAsync(h->arena + b.off, src, n, cudaMemcpyHostToDevice, s));
    return CFR_OK;
  };
  int rc;
  if ((rc = up(h->b_iset_slot, c.iset_slot.data(), 4 * (c.I + 1)))) return rc;
  if ((rc = up(h->b_iset_mem, c.iset_mem.data(), 4 * (c.I + 1)))) return rc;
  if ((rc = up(h->b_iset_vb, c.iset_vb.data(), 4 * c.I))) return rc;
  if ((rc = up(h->b_mem_vs, c.mem_vs.data(), 4 * c.n_dec))) return rc;
  if ((rc = up(h->b_ch_vb, c.ch_vb.data(), 4 * c.ch_vb.size()))) return rc;
  if ((rc = up(h->b_ch_nch, c.ch_nch.data(), 4 * c.ch_nch.size()))) return rc;
  if ((rc = up(h->b_ch_vs, c.ch_vs.data(), 4 * c.ch_vs.size()))) return rc;
  if ((rc = up(h->b_spec_slot, c.spec_slot_of.data(), 4 * c.A))) return rc;
  if ((rc = up(h->b_levels, h->levels.data(), sizeof(LevelWork) * c.D))) return rc;
  if ((rc = up(h->b_wide_vb, c.wide_vb.data(), 4 * c.n_wide))) return rc;
  if ((rc = up(h->b_wide_nch, c.wide_nch.data(), 4 * c.n_wide))) return rc;
  if ((rc = up(h->b_wide_vs, c.wide_vs.data(), 4 * c.n_wide))) return rc;
  if ((rc = up(h->b_wide_chunk, c.wide_chunk.data(), 4 * (c.n_wide + 1)))) return rc;
  if ((rc = up(h->b_int_slot, c.int_slot.data(), 4 * c.int_slot.size()))) return rc;
  if ((rc = up(h->b_int_mask, c.int_mask.data(), 4 * c.int_mask.size()))) return rc;
  if ((rc = up(h->b_int_cirank, c.int_cirank.data(), 4 * c.int_cirank.size()))) return rc;
  if ((rc = up(h->b_big_irank, c.big_irank.data(), 4 * c.big_irank.size()))) return rc;
  if ((rc = up(h->b_int_edge, c.int_edge.data(), 4 * c.int_edge.size()))) return rc;
  if ((rc = up(h->b_iset_rank, c.iset_rank.data(), 4 * c.iset_rank.size()))) return rc;
  if ((rc = up(h->b_mem_irank, c.mem_irank.data(), h->b_mem_irank.bytes))) return rc;
  if ((rc = up(h->b_wide_irank, c.wide_irank.data(), 4 * c.wide_irank.size()))) return rc;
  if ((rc = up(h->b_set_info, h->set_info.data(), sizeof(SetInfo) * h->set_info.size()))) return rc;
  if ((rc = up(h->b_stream_chunks, h->stream_chunks.data(), sizeof(StreamChunk) * h->stream_chunks.size()))) return rc;
  if (!h->stream_chunks.empty()) CK(prepare_bwd_stream());
  if ((rc = h->precision == CFR_P64 ? default_pull_grids<double>(h) : default_pull_grids<float>(h))) return rc;
  if (c.n_wide) CK(cudaMemsetAsync(h->arena + h->b_wide_cnt.off, 0, 4 * c.n_wide, s));
  CK(cudaMemsetAsync(h->arena + h->b_bar.off, 0, 16, s));
  CK(cudaMemsetAsync(h->arena + h->b_err.off, 0, 16, s));
  if (h->precision == CFR_P64) {
    if ((rc = init_state<double>(h, s))) return rc;
    if ((rc = init_values<double>(h, s))) return rc;
  } else {
    if ((rc = init_state<float>(h, s))) return rc;
    if ((rc = init_values<float>(h, s))) return rc;
  }
  CK(cudaStreamSynchronize(s));
  h->bound = true;
  return CFR_OK;
}

// ------------------------------------------------------------ iteration
// upd: the players whose sets update (bit 0 player 1, bit 1 player 2); the
// depth-0 launch of the pass that updates player 2 advances t.
// Streaming CTAs of the streaming backward of depth d: two per SM, never
// more than the depth has chunks.
static int stream_ctas(const cfr_handle *h, int d) {
  const int n = h->stream_c0[d + 1] - h->stream_c0[d];
  return std::max(1, std::min(n, 2 * device_sms()));
}

// Blocks of the backward launch of depth d (chance blocks, wide chunks, then
// the information-set work; the streaming form has only its CTAs over the
// depth's set and chance chunks).
static void bwd_blocks(const cfr_handle *h, int d, int *nb_ch, int *nb_wide, int *nb_is) {
  const LevelWork &w = h->levels[d];
  const int nch = d > 0 ? w.ch1 - w.ch0 : 0, nis = w.is1 - w.is0;  // a chance root is skipped
  const int lanes = h->level_lanes[d];
  // the streaming form sums its chance nodes in chunks of its own
  *nb_ch = nch > 0 && lanes != kStreamLanes ? grid_for(nch, kThreads) : 0;
  *nb_wide = d > 0 ? w.wc1 - w.wc0 : 0;
  if (lanes == kStreamLanes) *nb_is = nis > 0 ? stream_ctas(h, d) : 0;
  else *nb_is = nis > 0 ? grid_for(nis, kThreads / lanes) : 0;
}

// upd: the players whose sets update (bit 0 player 1, bit 1 player 2); the
// depth-0 launch of the pass that updates player 2 advances t.
template <typename T>
static int launch_bwd(cfr_handle *h, int d, cudaStream_t s, int upd = 3, bool pdl = false) {
  LevelWork w = h->levels[d];
  if (d == 0) {  // a chance root's value has no reader in an iteration (the best response sums its own)
    w.ch1 = w.ch0;
    w.wc1 = w.wc0;
  }
  int nb_ch, nb_wide, nb_is;
  bwd_blocks(h, d, &nb_ch, &nb_wide, &nb_is);
  const int lanes = h->level_lanes[d];
  if (lanes == kStreamLanes) {  // FP32 only (compile checks it); no wide chance nodes at this depth
    // with programmatic dependent launch the launch before a backward launch
    // of depth d < D - 1 is the backward launch of depth d + 1
    CK(launch_bwd_stream(h->maxa_tier, nb_is, s, game_view(h), state_view<float>(h), h->p<SetInfo>(h->b_set_info),
                         h->p<StreamChunk>(h->b_stream_chunks), h->stream_c0[d], h->stream_c0[d + 1], h->rule, upd,
                         h->p<int>(h->b_err), pdl, pdl && d + 1 < h->c.D));
    return CFR_OK;
  }
  // at least one block: the depth-0 launch also advances t
  CK(launch_bwd_level<T>(h->maxa_tier, lanes, std::max(1, nb_ch + nb_wide + nb_is), s, game_view(h), state_view<T>(h),
                         w, nb_ch, h->rule, upd, (d == 0 && (upd & 2)) ? 1 : 0, pdl));
  return CFR_OK;
}

// Programmatic dependent launch between the per-level kernels: on by
// choice, or by default in FP32 only (in FP64 the overlapped graph ran the
// card game 22% slower on one GB300, 10.4 against 8.5 ms per iteration).
static bool overlap_on(const cfr_handle *h) {
  if (h->opt.launch_overlap == CFR_OVERLAP_AUTO) return h->precision == CFR_P32;
  return h->opt.launch_overlap == CFR_OVERLAP_ON;
}

// One iteration's launches. Every launch but the first of the iteration may
// overlap its predecessor's tail (programmatic dependent launch).
template <typename T>
static int enqueue_iteration(cfr_handle *h, cudaStream_t s, bool first_overlaps = false) {
  const Compiled &c = h->c;
  GameView g = game_view(h);
  const int halves = h->order == CFR_ORDER_ALTERNATING ? 2 : 1;
  const bool ov = overlap_on(h);
  bool pdl = ov && first_overlaps;
  for (int hf = 0; hf < halves; ++hf) {
    const int upd = halves == 2 ? (1 << hf) : 3;
    for (int64_t d = 0; d < c.D; ++d) {
      if (g.int_edge && d + 1 >= c.D) continue;  // member order: no launch for the deepest depth
      int rc = launch_fwd<T>(h, d, s, g, h->p<T>(h->b_sigma), h->p<vec2_t<T>>(h->b_reach), pdl);
      if (rc) return rc;
      pdl = ov;
    }
    for (int64_t d = c.D - 1; d >= 0; --d) {
      int rc = launch_bwd<T>(h, (int)d, s, upd, pdl);
      if (rc) return rc;
      pdl = ov;
    }
  }
  return CFR_OK;
}

// Blocks of the persistent form: enough for the widest depth, never more than
// can be co-resident (computed once per lane count).
template <typename T>
static int ensure_persist_grid(cfr_handle *h, cudaStream_t s) {
  if (h->persist_grid != 0) return CFR_OK;
  const int L = h->persist_lanes;
  PersistArgs<T> a{};
  int dev = 0, nsm = 0, per_sm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CK(launch_persistent<T>(h->maxa_tier, L, 0, s, a, &per_sm));
  int64_t cap = (int64_t)nsm * std::max(per_sm, 1);
  if (h->opt.persistent_ctas > 0) cap = std::min<int64_t>(cap, h->opt.persistent_ctas);
  int64_t need = 1;
  for (const LevelWork &w : h->levels) {
    need = std::max<int64_t>(need, (w.ie - w.ib + 4 * kThreads - 1) / (4 * kThreads));
    need = std::max<int64_t>(need, (w.ch1 - w.ch0 + kThreads - 1) / kThreads);
    need = std::max<int64_t>(need, ((int64_t)(w.is1 - w.is0) * L + kThreads - 1) / kThreads);
    need = std::max<int64_t>(need, w.wc1 - w.wc0);
  }
  h->persist_grid = (int)std::max<int64_t>(1, std::min(need, cap));
  return CFR_OK;
}

template <typename T>
static int launch_persistent_form(cfr_handle *h, int64_t n, cudaStream_t s) {
  const int L = h->persist_lanes;
  PersistArgs<T> a;
  a.g = game_view(h);
  a.st = state_view<T>(h);
  a.lw = h->p<LevelWork>(h->b_levels);
  a.D = (int)h->c.D;
  a.rule = h->rule;
  a.order = h->order;
  a.n_iter = n;
  unsigned *bar = h->p<unsigned>(h->b_bar);
  a.bar.count = bar;
  a.bar.gen = bar + 1;
  a.bar.err = h->p<int>(h->b_err);
  a.bar.spin_limit = h->opt.barrier_spin_limit > 0 ? h->opt.barrier_spin_limit : (int64_t)20000000;
  int rc = ensure_persist_grid<T>(h, s);
  if (rc) return rc;
  a.bar.expected = (unsigned)h->persist_grid + (unsigned)h->test_missing_arrivals;
  CK(cudaMemsetAsync(bar, 0, 4, s));  // arrivals (a timed-out launch leaves them set)
  CK(launch_persistent<T>(h->maxa_tier, L, h->persist_grid, s, a, nullptr));
  return CFR_OK;
}

// Captures `iters` iterations into an executable graph. A refused capture
// (or instantiation) warns once per handle and sets *failed.
template <typename T>
static int capture_iterations(cfr_handle *h, int iters, cudaGraphExec_t *out, bool *failed, int64_t *kernels) {
  *failed = false;
  if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = CFR_OK;
  for (int i = 0; i < iters && rc == CFR_OK; ++i) rc = enqueue_iteration<T>(h, h->cap_stream, i > 0);
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e == cudaSuccess && h->test_fail_capture) {  // test hook: the same path as a refused capture
    cudaGraphDestroy(graph);
    graph = nullptr;
    e = cudaErrorStreamCaptureUnsupported;
  }
  if (e == cudaSuccess) {  // count the kernel nodes (the launch-count gate)
    size_t nn = 0;
    e = cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess && nn) e = cudaGraphGetNodes(graph, nodes.data(), &nn);
    int64_t nk = 0;
    for (size_t i = 0; i < nn && e == cudaSuccess; ++i) {
      cudaGraphNodeType ty;
      e = cudaGraphNodeGetType(nodes[i], &ty);
      if (e == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++nk;
    }
    *kernels = nk;
  }
  if (e == cudaSuccess) {
    e = cudaGraphInstantiate(out, graph, 0);
    if (e != cudaSuccess) *out = nullptr;
  }
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    // capture failed: warn once, fall back to per-level launches (same kernels, same order)
    if (!h->capture_warned) {
      fprintf(stderr, "cfr: graph capture failed (%s); using per-level launches\n", cudaGetErrorString(e));
      fflush(stderr);
      h->capture_warned = true;
    }
    cudaGetLastError();
    *failed = true;
  }
  return CFR_OK;
}

static void drop_graphs(cfr_handle *h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->gexec_k) cudaGraphExecDestroy(h->gexec_k);
  h->gexec = nullptr;
  h->gexec_k = nullptr;
}

template <typename T>
static int iterate_t(cfr_handle *h, int64_t n, cudaStream_t s) {
  if (h->c.D == 0) {  // root is terminal: nothing to update but the counter
    bump_t_kernel<<<1, 1, 0, s>>>(h->p<long long>(h->b_t), n);
    CK(cudaGetLastError());
    return CFR_OK;
  }
  if (h->exec_form == CFR_EXEC_LEVELS) {
    for (int64_t i = 0; i < n; ++i) {
      int rc = enqueue_iteration<T>(h, s, i > 0);
      if (rc) return rc;
    }
    return CFR_OK;
  }
  if (h->exec_form == CFR_EXEC_PERSISTENT) return launch_persistent_form<T>(h, n, s);
  // graph form: k iterations per graph (k = graph_iters) replayed n / k
  // times, and a one-iteration graph for the rest; both captured on first
  // use (cfr_bind drops them, so a replay always refers to the bound arena)
  const int k = std::max(1, h->opt.graph_iters);
  const int64_t nk = k > 1 ? n / k : 0, n1 = n - nk * k;
  bool failed = false;
  if (nk > 0 && !h->gexec_k) {
    int rc = capture_iterations<T>(h, k, &h->gexec_k, &failed, &h->graph_k_kernels);
    if (rc) return rc;
  }
  if (!failed && n1 > 0 && !h->gexec) {
    int rc = capture_iterations<T>(h, 1, &h->gexec, &failed, &h->graph_kernels);
    if (rc) return rc;
  }
  if (failed) {
    drop_graphs(h);
    h->exec_form = CFR_EXEC_LEVELS;
    return iterate_t<T>(h, n, s);
  }
  for (int64_t i = 0; i < nk; ++i) CK(cudaGraphLaunch(h->gexec_k, s));
  for (int64_t i = 0; i < n1; ++i) CK(cudaGraphLaunch(h->gexec, s));
  return CFR_OK;
}

extern "C" int cfr_iterate(cfr_handle *h, int64_t n, void *stream) {
  if (!h) return set_err(CFR_ERR_ARG, "cfr_iterate: null handle");
  if (n < 0) return set_err(CFR_ERR_ARG, "cfr_iterate: negative n");
  if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "cfr_iterate: call cfr_bind first");
  if (n == 0) return CFR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = h->precision == CFR_P64 ? iterate_t<double>(h, n, s) : iterate_t<float>(h, n, s);
  if (rc == CFR_OK) h->iteration_host += n;
  return rc;
}

extern "C" int cfr_synchronize(cfr_handle *h, void *stream) {
  if (!h) return set_err(CFR_ERR_ARG, "cfr_synchronize: null handle");
  if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "cfr_synchronize: not bound");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaStreamSynchronize(s));
  int err = 0;
  CK(cudaMemcpy(&err, h->arena + h->b_err.off, 4, cudaMemcpyDeviceToHost));
  if (err) {
    CK(cudaMemset(h->arena + h->b_err.off, 0, 4));
    return set_err(CFR_ERR_TIMEOUT, "a bounded wait in a kernel gave up (a grid barrier of the persistent kernel, or a "
                   "staged copy of the streaming backward); the state is undefined until cfr_reset");
  }
  return CFR_OK;
}

// ------------------------------------------------------------- read-out
static int deliver(cfr_handle *h, const double *dev_compiled, double *out, int on_device, cudaStream_t s) {
  const Compiled &c = h->c;
  if (c.A == 0) return CFR_OK;
  double *dst = on_device ? out : h->p<double>(h->b_out);
  permute_kernel<<<grid_for(c.A, kThreads), kThreads, 0, s>>>(h->p<int32_t>(h->b_spec_slot), dev_compiled, dst, (int32_t)c.A);
  CK(cudaGetLastError());
  if (!on_device) {
    CK(cudaMemcpyAsync(out, dst, 8 * c.A, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return CFR_OK;
}

extern "C" int cfr_avg_strategy(cfr_handle *h, double *out, int on_device, void *stream) {
  if (!h || (!out && h->c.A > 0)) return set_err(CFR_ERR_ARG, "cfr_avg_strategy: null argument");
  if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "cfr_avg_strategy: not bound");
  cudaStream_t s = (cudaStream_t)stream;
  const Compiled &c = h->c;
  if (c.I == 0) return CFR_OK;
  avg_normalize_kernel<<<grid_for(c.I, kThreads), kThreads, 0, s>>>(h->p<int32_t>(h->b_iset_slot), (int32_t)c.I,
                                                                     h->p<double>(h->b_avg), h->p<double>(h->b_sbs));
  CK(cudaGetLastError());
  return deliver(h, h->p<double>(h->b_sbs), out, on_device, s);
}

extern "C" int cfr_current_strategy(cfr_handle *h, double *out, int on_device, void *stream) {
  if (!h || (!out && h->c.A > 0)) return set_err(CFR_ERR_ARG, "cfr_current_strategy: null argument");
  if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "cfr_current_strategy: not bound");
  cudaStream_t s = (cudaStream_t)stream;
  const Compiled &c = h->c;
  if (c.A == 0) return CFR_OK;
  double *tmp = h->p<double>(h->b_sbs);
  if (h->precision == CFR_P64) CK(cudaMemcpyAsync(tmp, h->p<double>(h->b_sigma), 8 * c.A, cudaMemcpyDeviceToDevice, s));
  else {
    to_double_kernel<float><<<grid_for(c.A, kThreads), kThreads, 0, s>>>(h->p<float>(h->b_sigma), tmp, (int32_t)c.A);
    CK(cudaGetLastError());
  }
  return deliver(h, tmp, out, on_device, s);
}

static int launch_br(cfr_handle *h, int d, cudaStream_t s) {
  const LevelWork &w = h->levels[d];
  const int L = std::min(h->level_lanes[d], 32);  // best response: lane groups of at most a warp
  const int nch = w.ch1 - w.ch0, nis = w.is1 - w.is0;
  const int nb_ch = nch > 0 ? grid_for(nch, kThreads) : 0;
  const int nb_is = nis > 0 ? grid_for(nis, kThreads / L) : 0;
  const int nb_wide = w.wc1 - w.wc0;
  CK(launch_br_level(h->maxa_tier, L, std::max(1, nb_ch + nb_wide + nb_is), s, game_view(h), h->p<double2>(h->b_reach2),
                     h->p<double>(h->b_sbs), h->p<double2>(h->b_vb), h->p<double>(h->b_vavg), w, nb_ch));
  return CFR_OK;
}

extern "C" int cfr_exploitability(cfr_handle *h, double *out_expl, double *out_br, void *stream) {
  if (!h || !out_expl) return set_err(CFR_ERR_ARG, "cfr_exploitability: null argument");
  if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "cfr_exploitability: not bound");
  cudaStream_t s = (cudaStream_t)stream;
  const Compiled &c = h->c;
  GameView g = game_view(h);
  if (c.I > 0)
    avg_normalize_kernel<<<grid_for(c.I, kThreads), kThreads, 0, s>>>(h->p<int32_t>(h->b_iset_slot), (int32_t)c.I,
                                                                       h->p<double>(h->b_avg), h->p<double>(h->b_sbs));
  CK(cudaGetLastError());
  for (int64_t d = 0; d < c.D; ++d) {
    int rc = launch_fwd<double>(h, d, s, g, h->p<double>(h->b_sbs), h->p<double2>(h->b_reach2));
    if (rc) return rc;
  }
  for (int64_t d = c.D - 1; d >= 0; --d) {
    int rc = launch_br(h, (int)d, s);
    if (rc) return rc;
  }
  double root[3];
  const int64_t rs = c.N - 1;  // the root's value slot
  CK(cudaMemcpyAsync(root, h->p<double2>(h->b_vb) + rs, 16, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(root + 2, h->p<double>(h->b_vavg) + rs, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *out_expl = 0.5 * (root[0] - root[1]);
  if (out_br) { out_br[0] = root[0]; out_br[1] = root[1]; out_br[2] = root[2]; }
  return CFR_OK;
}

// ------------------------------------------------------------- lifecycle
extern "C" int cfr_reset(cfr_handle *h, void *stream) {
  if (!h) return set_err(CFR_ERR_ARG, "cfr_reset: null handle");
  if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "cfr_reset: not bound");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemsetAsync(h->arena + h->b_err.off, 0, 16, s));
  if (h->c.n_wide) CK(cudaMemsetAsync(h->arena + h->b_wide_cnt.off, 0, 4 * h->c.n_wide, s));
  return h->precision == CFR_P64 ? init_state<double>(h, s) : init_state<float>(h, s);
}

extern "C" int cfr_set_payoffs(cfr_handle *h, const double *payoff, void *stream) {
  if (!h || !payoff) return set_err(CFR_ERR_ARG, "cfr_set_payoffs: null argument");
  if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "cfr_set_payoffs: not bound");
  Compiled &c = h->c;
  for (int64_t x = 0; x < c.N; ++x)
    if (c.child_begin[x] == c.child_begin[x + 1] && !std::isfinite(payoff[c.spec_of_new[x]]))
      return set_err(CFR_ERR_ARG, "cfr_set_payoffs: non-finite payoff");
  for (int64_t x = 0; x < c.N; ++x)
    if (c.child_begin[x] == c.child_begin[x + 1]) {
      c.u[x] = payoff[c.spec_of_new[x]];
      c.tmpl[x] = c.pc[x] * c.u[x];
      c.tmpl_vs[c.vslot[x]] = c.tmpl[x];
    }
  cudaStream_t s = (cudaStream_t)stream;
  int rc = h->precision == CFR_P64 ? init_values<double>(h, s) : init_values<float>(h, s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  return CFR_OK;
}

extern "C" int cfr_set_root_chance(cfr_handle *h, const double *prob, int64_t n, void *stream) {
  if (!h || (!prob && n > 0)) return set_err(CFR_ERR_ARG, "cfr_set_root_chance: null argument");
  Compiled &c = h->c;
  if (c.N == 0 || c.child_begin[1] == c.child_begin[0] || c.node_slot[0] >= 0)
    return set_err(CFR_ERR_UNSUPPORTED, "cfr_set_root_chance: the root is not a chance node");
  const int64_t nch = c.child_begin[1] - c.child_begin[0];
  if (n != nch) return set_err(CFR_ERR_ARG, "cfr_set_root_chance: the root has %lld children, got %lld", (long long)nch, (long long)n);
  for (int64_t k = 0; k < n; ++k)
    if (!std::isfinite(prob[k]) || prob[k] < 0.0) return set_err(CFR_ERR_ARG, "cfr_set_root_chance: probability %lld is negative or not finite", (long long)k);
  for (int64_t k = 0; k < n; ++k) c.edge_p[c.child_begin[0] + k] = prob[k];
  fold_chance(c);
  if (!h->bound) return CFR_OK;  // cfr_bind uploads the new template
  cudaStream_t s = (cudaStream_t)stream;
  int rc = h->precision == CFR_P64 ? init_values<double>(h, s) : init_values<float>(h, s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  return CFR_OK;
}

extern "C" int cfr_get_state(cfr_handle *h, double *R, double *avg, int64_t *t, void *stream) {
  if (!h || ((!R || !avg) && h->c.A > 0) || !t) return set_err(CFR_ERR_ARG, "cfr_get_state: null argument");
  if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "cfr_get_state: not bound");
  cudaStream_t s = (cudaStream_t)stream;
  const Compiled &c = h->c;
  std::vector<double> r(c.A), a(c.A);
  long long tt = 0;
  if (c.A) {
    CK(cudaMemcpyAsync(r.data(), h->p<double>(h->b_R), 8 * c.A, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(a.data(), h->p<double>(h->b_avg), 8 * c.A, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaMemcpyAsync(&tt, h->p<long long>(h->b_t), 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int64_t q = 0; q < c.A; ++q) { R[c.spec_slot_of[q]] = r[q]; avg[c.spec_slot_of[q]] = a[q]; }
  *t = tt;
  return CFR_OK;
}

extern "C" int cfr_set_state(cfr_handle *h, const double *R, const double *avg, int64_t t, void *stream) {
  if (!h || ((!R || !avg) && h->c.A > 0) || t < 0) return set_err(CFR_ERR_ARG, "cfr_set_state: bad argument");
  if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "cfr_set_state: not bound");
  cudaStream_t s = (cudaStream_t)stream;
  const Compiled &c = h->c;
  std::vector<double> r(c.A), a(c.A);
  for (int64_t q = 0; q < c.A; ++q) { r[q] = R[c.spec_slot_of[q]]; a[q] = avg[c.spec_slot_of[q]]; }
  long long tt = t;
  if (c.A) {
    CK(cudaMemcpyAsync(h->p<double>(h->b_R), r.data(), 8 * c.A, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->p<double>(h->b_avg), a.data(), 8 * c.A, cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemcpyAsync(h->p<long long>(h->b_t), &tt, 8, cudaMemcpyHostToDevice, s));
  if (c.I) {
    if (h->precision == CFR_P64)
      rm_kernel<double><<<grid_for(c.I, kThreads), kThreads, 0, s>>>(h->p<int32_t>(h->b_iset_slot), (int32_t)c.I, h->p<double>(h->b_R), h->p<double>(h->b_sigma));
    else
      rm_kernel<float><<<grid_for(c.I, kThreads), kThreads, 0, s>>>(h->p<int32_t>(h->b_iset_slot), (int32_t)c.I, h->p<double>(h->b_R), h->p<float>(h->b_sigma));
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(s));
  h->iteration_host = t;
  return CFR_OK;
}

extern "C" int cfr_export_array(const cfr_handle *h, int which, void *out, int64_t capacity, int64_t *count) {
  if (!h || !count) return set_err(CFR_ERR_ARG, "cfr_export_array: null argument");
  const Compiled &c = h->c;
  const void *src = nullptr;
  int64_t n = 0;
  size_t esz = 4;
  switch (which) {
    case 0: src = c.child_begin.data(); n = (int64_t)c.child_begin.size(); break;
    case 1: src = c.node_slot.data(); n = (int64_t)c.node_slot.size(); break;
    case 2: src = c.level_begin.data(); n = (int64_t)c.level_begin.size(); break;
    case 3: src = c.iset_slot.data(); n = (int64_t)c.iset_slot.size(); break;
    case 4: src = c.iset_mem.data(); n = (int64_t)c.iset_mem.size(); break;
    case 5: src = c.mem_node.data(); n = (int64_t)c.mem_node.size(); break;
    case 6: src = c.chance_list.data(); n = (int64_t)c.chance_list.size(); break;
    case 7: src = c.level_chance.data(); n = (int64_t)c.level_chance.size(); break;
    case 8: src = c.level_iset.data(); n = (int64_t)c.level_iset.size(); break;
    case 9: src = c.new_of_spec.data(); n = (int64_t)c.new_of_spec.size(); break;
    case 10: src = c.tmpl.data(); n = (int64_t)c.tmpl.size(); esz = 8; break;
    case 11: src = c.spec_slot_of.data(); n = (int64_t)c.spec_slot_of.size(); break;
    case 12: src = h->level_lanes.data(); n = (int64_t)h->level_lanes.size(); break;
    case 13: src = c.int_slot.data(); n = (int64_t)c.int_slot.size(); break;
    case 14: src = c.int_mask.data(); n = (int64_t)c.int_mask.size(); break;
    case 15: src = c.int_cirank.data(); n = (int64_t)c.int_cirank.size(); break;
    case 16: src = c.big_irank.data(); n = (int64_t)c.big_irank.size(); break;
    case 17: src = c.mem_irank.data(); n = (int64_t)c.mem_irank.size(); break;
    case 18: src = c.level_int.data(); n = (int64_t)c.level_int.size(); break;
    case 19: src = c.vslot.data(); n = (int64_t)c.vslot.size(); break;
    case 20: src = c.iset_vb.data(); n = (int64_t)c.iset_vb.size(); break;
    case 21: src = c.mem_vs.data(); n = (int64_t)c.mem_vs.size(); break;
    case 22: src = c.ch_vb.data(); n = (int64_t)c.ch_vb.size(); break;
    case 23: src = c.ch_nch.data(); n = (int64_t)c.ch_nch.size(); break;
    case 24: src = c.ch_vs.data(); n = (int64_t)c.ch_vs.size(); break;
    case 25: src = c.wide_vb.data(); n = (int64_t)c.wide_vb.size(); break;
    case 26: src = c.wide_nch.data(); n = (int64_t)c.wide_nch.size(); break;
    case 27: src = c.wide_vs.data(); n = (int64_t)c.wide_vs.size(); break;
    case 28: src = c.tmpl_vs.data(); n = (int64_t)c.tmpl_vs.size(); esz = 8; break;
    case 29: src = c.int_edge.data(); n = (int64_t)c.int_edge.size(); break;
    case 30: src = c.iset_rank.data(); n = (int64_t)c.iset_rank.size(); break;
    case 31: src = c.level_tiled.data(); n = (int64_t)c.level_tiled.size(); break;
    case 32: src = h->set_info.data(); n = 8 * (int64_t)h->set_info.size(); break;
    case 33: src = h->stream_chunks.data(); n = 16 * (int64_t)h->stream_chunks.size(); break;
    case 34: src = h->stream_c0.data(); n = (int64_t)h->stream_c0.size(); break;
    case 35: src = h->stream_ok.data(); n = (int64_t)h->stream_ok.size(); break;
    case 36: src = h->pull_grid.data(); n = (int64_t)h->pull_grid.size(); break;
    default: return set_err(CFR_ERR_ARG, "cfr_export_array: unknown array %d", which);
  }
  *count = n;
  if (!out) return CFR_OK;
  if (capacity < n) return set_err(CFR_ERR_ARG, "cfr_export_array: capacity %lld < %lld", (long long)capacity, (long long)n);
  if (n) memcpy(out, src, esz * (size_t)n);
  return CFR_OK;
}

extern "C" int cfr_debug_set(cfr_handle *h, int key, int64_t value) {
  if (!h) return set_err(CFR_ERR_ARG, "cfr_debug_set: null handle");
  if (key == CFR_DEBUG_BARRIER_MISSING_ARRIVALS) {
    if (value < 0 || value > 1024) return set_err(CFR_ERR_ARG, "cfr_debug_set: bad value");
    h->test_missing_arrivals = (int)value;
    return CFR_OK;
  }
  if (key == CFR_DEBUG_FAIL_GRAPH_CAPTURE) {
    if (value != 0 && value != 1) return set_err(CFR_ERR_ARG, "cfr_debug_set: bad value");
    h->test_fail_capture = (int)value;
    return CFR_OK;
  }
  if (key == CFR_DEBUG_STREAM_STALL) {  // the second word of the error array, read by the streaming kernel
    if (value != 0 && value != 1) return set_err(CFR_ERR_ARG, "cfr_debug_set: bad value");
    if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "cfr_debug_set: the stall flag needs a bound handle");
    const int v = (int)value;
    CK(cudaMemcpy(h->arena + h->b_err.off + 4, &v, 4, cudaMemcpyHostToDevice));
    return CFR_OK;
  }
  return set_err(CFR_ERR_ARG, "cfr_debug_set: unknown key %d", key);
}

extern "C" int cfr_level_bytes(const cfr_handle *h, int d, int64_t *fwd, int64_t *bwd) {
  if (!h || !fwd || !bwd) return set_err(CFR_ERR_ARG, "cfr_level_bytes: null argument");
  const Compiled &c = h->c;
  if (d < 0 || d >= c.D) return set_err(CFR_ERR_ARG, "cfr_level_bytes: level out of range");
  const int64_t T = h->precision == CFR_P64 ? 8 : 4;
  int64_t e = c.level_begin[d + 2] - c.level_begin[d + 1];  // children = next level
  const int64_t nint = c.level_int[d + 1] - c.level_int[d];
  const int64_t nint_kids = (d + 1 < c.D) ? c.level_int[d + 2] - c.level_int[d + 1] : 0;
  const int64_t i0 = c.level_iset[2 * d], i1 = c.level_iset[2 * d + 2];
  const int64_t sets = i1 - i0;
  const int64_t slots = c.iset_slot[i1] - c.iset_slot[i0];
  const int64_t dec = c.iset_mem[i1] - c.iset_mem[i0];
  int64_t nch = (c.level_chance[d + 1] - c.level_chance[d]) + (c.level_wide[d + 1] - c.level_wide[d]);
  if (d == 0 && nch > 0) nch = e = 0;  // a chance root's sum is not done in an iteration
  if (!c.int_edge.empty()) {  // member order: the launch of depth d fills depth d + 1 by pulling
    *fwd = d + 1 < c.D ? 8 * nint_kids + 2 * T * c.level_pull_parents[d] + 2 * T * nint_kids + T * slots : 0;
    *bwd = 12 * sets + (32 + 2 * T) * slots + (4 + 3 * T) * dec + (12 + T) * nch + T * e;
    return CFR_OK;
  }
  int64_t big = 0;  // child lists of nodes with more than 31 children
  for (int64_t q = c.level_int[d]; q < c.level_int[d + 1]; ++q)
    if (c.int_mask[q] & kBigNode) big += 1 + c.big_irank[c.int_cirank[q]];
  *fwd = 12 * nint + 2 * T * nint + 2 * T * nint_kids + T * slots + 4 * big;
  *bwd = 12 * sets + (32 + 2 * T) * slots + (8 + 3 * T) * dec + (12 + T) * nch + T * e;
  return CFR_OK;
}

// One iteration with an event pair around every launch; under alternating
// updates the two halves' times of a launch are added.
template <typename T>
static int profile_t(cfr_handle *h, double *fwd_ms, double *bwd_ms, cudaStream_t s) {
  const Compiled &c = h->c;
  const int halves = h->order == CFR_ORDER_ALTERNATING ? 2 : 1;
  std::vector<cudaEvent_t> ev(4 * c.D * halves + 2, nullptr);
  for (auto &e : ev) CK(cudaEventCreate(&e));
  GameView g = game_view(h);
  int rc = CFR_OK;
  for (int hf = 0; hf < halves && rc == CFR_OK; ++hf) {
    const int upd = halves == 2 ? (1 << hf) : 3;
    cudaEvent_t *e = ev.data() + 4 * c.D * hf;
    for (int64_t d = 0; d < c.D && rc == CFR_OK; ++d) {
      CK(cudaEventRecord(e[2 * d], s));
      rc = launch_fwd<T>(h, d, s, g, h->p<T>(h->b_sigma), h->p<vec2_t<T>>(h->b_reach));
      CK(cudaEventRecord(e[2 * d + 1], s));
    }
    for (int64_t d = c.D - 1; d >= 0 && rc == CFR_OK; --d) {
      CK(cudaEventRecord(e[2 * c.D + 2 * d], s));
      rc = launch_bwd<T>(h, (int)d, s, upd);
      CK(cudaEventRecord(e[2 * c.D + 2 * d + 1], s));
    }
  }
  CK(cudaStreamSynchronize(s));
  for (int64_t d = 0; d < c.D; ++d) {
    fwd_ms[d] = 0.0;
    bwd_ms[d] = 0.0;
    for (int hf = 0; hf < halves; ++hf) {
      cudaEvent_t *e = ev.data() + 4 * c.D * hf;
      float a = 0.f, b = 0.f;
      CK(cudaEventElapsedTime(&a, e[2 * d], e[2 * d + 1]));
      CK(cudaEventElapsedTime(&b, e[2 * c.D + 2 * d], e[2 * c.D + 2 * d + 1]));
      fwd_ms[d] += a;
      bwd_ms[d] += b;
    }
  }
  for (auto &e : ev) cudaEventDestroy(e);
  if (rc == CFR_OK) h->iteration_host += 1;
  return rc;
}

extern "C" int cfr_profile_iteration(cfr_handle *h, double *fwd_ms, double *bwd_ms, void *stream) {
  if (!h || ((!fwd_ms || !bwd_ms) && h->c.D > 0)) return set_err(CFR_ERR_ARG, "cfr_profile_iteration: null argument");
  if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "cfr_profile_iteration: not bound");
  if (h->c.D == 0) return cfr_iterate(h, 1, stream);
  cudaStream_t s = (cudaStream_t)stream;
  return h->precision == CFR_P64 ? profile_t<double>(h, fwd_ms, bwd_ms, s) : profile_t<float>(h, fwd_ms, bwd_ms, s);
}

// ---------------------------------------------------------------------------
// Allocation-free iteration (no counterpart in the paper).
//
// Some callers cannot allocate device memory at the moment they want to run
// iterations: serving loops whose device memory is carved out once at
// start-up, or host code that embeds the library without owning the device
// allocator. cfr_iterate_noalloc serves them: it runs
// the persistent kernel with its per-iteration scratch (both reach lanes, the
// node values, wide-node partial sums and the grid-barrier words) placed in
// one file-scope device array of fixed size, so the call itself allocates
// nothing. The bound arena still holds the compiled game and the solver state
// (regrets, average, strategy, t), which are this call's inputs and outputs.
constexpr size_t kNoAllocScratchBytes = size_t(12) << 20;  // 12 MiB per GPU, held until exit
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[256];  // device address of the array, per device ordinal

// Host code may not use the array's name as a device address: resolve it
// once per device, with that device current.
static int noalloc_scratch(void **out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return set_err(CFR_ERR_DEVICE, "cfr_iterate_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return CFR_OK;
}

// Every call starts from a clean scratch: value slots from the template,
// root reach (1, 1), wide-node tickets and barrier words at zero.
template <typename T>
__global__ void noalloc_init_kernel(const double *tmpl_vs, int32_t N, T *v, vec2_t<T> *reach, unsigned *wide_cnt,
                                    int32_t n_wide, unsigned *bar) {
  const int32_t stride = gridDim.x * blockDim.x;
  const int32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  for (int32_t h = tid; h < N; h += stride) v[h] = (T)tmpl_vs[h];
  for (int32_t i = tid; i < n_wide; i += stride) wide_cnt[i] = 0u;
  if (tid == 0) {
    vec2_t<T> one;
    one.x = T(1); one.y = T(1);
    reach[0] = one;
    bar[0] = 0u; bar[1] = 0u; bar[2] = 0u;
  }
}

template <typename T>
static int iterate_noalloc_t(cfr_handle *h, int64_t n, cudaStream_t s) {
  const Compiled &c = h->c;
  size_t off_v = align_up(2 * sizeof(T) * (size_t)std::max<int64_t>(c.n_int, 1));
  size_t off_part = off_v + align_up(sizeof(T) * (size_t)c.N);
  size_t off_cnt = off_part + align_up(3 * 8 * (size_t)c.wide_chunk.back());
  size_t off_bar = off_cnt + align_up(4 * (size_t)c.n_wide);
  const size_t need = off_bar + 256;
  if (need > kNoAllocScratchBytes)
    return set_err(CFR_ERR_ARG, "cfr_iterate_noalloc: the game needs %zu bytes of scratch, the static limit is %zu "
                   "(about %lld nodes in FP64, %lld in FP32)", need, kNoAllocScratchBytes,
                   (long long)(kNoAllocScratchBytes / 24), (long long)(kNoAllocScratchBytes / 12));
  void *base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc) return rc;
  char *sb = (char *)base;
  PersistArgs<T> a;
  a.g = game_view(h);
  a.g.wide_part = (double *)(sb + off_part);
  a.g.wide_cnt = (unsigned *)(sb + off_cnt);
  a.st = state_view<T>(h);
  a.st.reach = (vec2_t<T> *)sb;
  a.st.v = (T *)(sb + off_v);
  a.lw = h->p<LevelWork>(h->b_levels);
  a.D = (int)c.D;
  a.rule = h->rule;
  a.order = h->order;
  a.n_iter = n;
  unsigned *bar = (unsigned *)(sb + off_bar);
  a.bar.count = bar;
  a.bar.gen = bar + 1;
  a.bar.err = (int *)(bar + 2);
  a.bar.spin_limit = h->opt.barrier_spin_limit > 0 ? h->opt.barrier_spin_limit : (int64_t)20000000;
  // the persistent form's grid (computed once per lane count; allocates nothing)
  if ((rc = ensure_persist_grid<T>(h, s))) return rc;
  const int grid = h->persist_grid;
  a.bar.expected = (unsigned)grid;
  noalloc_init_kernel<T><<<grid_for(c.N, kThreads), kThreads, 0, s>>>(
      h->p<double>(h->b_tmpl), (int32_t)c.N, a.st.v, a.st.reach, a.g.wide_cnt,
      (int32_t)c.n_wide, bar);
  CK(cudaGetLastError());
  CK(launch_persistent<T>(h->maxa_tier, h->persist_lanes, grid, s, a, nullptr));
  int err = 0;
  CK(cudaMemcpyAsync(&err, bar + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (err) return set_err(CFR_ERR_TIMEOUT, "cfr_iterate_noalloc: a grid barrier gave up waiting; the state is undefined until cfr_reset");
  return CFR_OK;
}

extern "C" int cfr_iterate_noalloc(cfr_handle *h, int64_t n, void *stream) {
  if (!h) return set_err(CFR_ERR_ARG, "cfr_iterate_noalloc: null handle");
  if (n < 0) return set_err(CFR_ERR_ARG, "cfr_iterate_noalloc: negative n");
  if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "cfr_iterate_noalloc: call cfr_bind first");
  if (n == 0) return CFR_OK;
  if (h->c.D == 0) return set_err(CFR_ERR_UNSUPPORTED, "cfr_iterate_noalloc: the root is terminal; use cfr_iterate");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = h->precision == CFR_P64 ? iterate_noalloc_t<double>(h, n, s) : iterate_noalloc_t<float>(h, n, s);
  if (rc == CFR_OK) h->iteration_host += n;
  return rc;
}

// Autotuner: per depth, time the backward launch with every lane count the
// action tier has kernels for and keep the fastest; for the persistent form,
// time whole persistent iterations per lane count. Trial launches change the
// state, so the call ends with the state reset (as cfr_reset).
// ------------------------------------------------------------ launch floor
// The iteration's launch structure with no work in it: the same launches
// (2D, or 2D - 1 in member order; same grid sizes) of an empty kernel
// captured in one graph, and one cooperative launch of an empty kernel with
// the persistent form's grid and its 2D grid barriers per iteration.
static __global__ void empty_level_kernel() { pdl_enter(); }

static __global__ void __launch_bounds__(kThreads) empty_persistent_kernel(Barrier bar, int n_sync, long long n_iter) {
  for (long long it = 0; it < n_iter; ++it)
    for (int k = 0; k < n_sync; ++k)
      if (!grid_sync(bar)) return;
}

extern "C" int cfr_launch_floor(cfr_handle *h, int64_t n, void *stream, double *graph_ms, double *persistent_ms) {
  if (!h || !graph_ms || !persistent_ms) return set_err(CFR_ERR_ARG, "cfr_launch_floor: null argument");
  if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "cfr_launch_floor: call cfr_bind first");
  if (n < 1 || n > 1000000) return set_err(CFR_ERR_ARG, "cfr_launch_floor: n must be in [1, 1e6]");
  *graph_ms = 0.0;
  *persistent_ms = 0.0;
  const Compiled &c = h->c;
  if (c.D == 0) return CFR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> grids;
  for (int64_t d = 0; d < c.D; ++d) {
    const LevelWork &w = h->levels[d];
    if (c.int_edge.empty()) grids.push_back(grid_for((w.ie - w.ib + 3) / 4, kThreads) + (w.wc1 - w.wc0));
    else if (d + 1 < c.D)  // member order: the launch of depth d pulls depth d + 1
      grids.push_back(h->pull_grid[d] > 0 ? h->pull_grid[d] : pull_need(h, d));
  }
  for (int64_t d = c.D - 1; d >= 0; --d) {
    int nb_ch, nb_wide, nb_is;
    bwd_blocks(h, (int)d, &nb_ch, &nb_wide, &nb_is);
    grids.push_back(std::max(1, nb_ch + nb_wide + nb_is));
  }
  if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t ge = nullptr;
  const int halves = h->order == CFR_ORDER_ALTERNATING ? 2 : 1;
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  bool pdl = false;  // the same programmatic dependencies as the iteration's launches
  for (int hf = 0; hf < halves; ++hf)
    for (int gsz : grids) {
      CK(launch_k(empty_level_kernel, std::max(gsz, 1), kThreads, 0, h->cap_stream, pdl));
      pdl = overlap_on(h);
    }
  CK(cudaStreamEndCapture(h->cap_stream, &graph));
  cudaError_t e = cudaGraphInstantiate(&ge, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return set_err(CFR_ERR_DEVICE, "cfr_launch_floor: %s", cudaGetErrorString(e));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = CFR_OK;
  float ms = 0.f;
  e = cudaGraphLaunch(ge, s);  // warm
  for (int64_t i = 0; i < n && e == cudaSuccess; ++i) {
    if (i == 0) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, s);
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaGraphExecDestroy(ge);
  if (e != cudaSuccess) rc = set_err(CFR_ERR_DEVICE, "cfr_launch_floor: %s", cudaGetErrorString(e));
  if (rc == CFR_OK) {
    *graph_ms = (double)ms / (double)n;
    rc = h->precision == CFR_P64 ? ensure_persist_grid<double>(h, s) : ensure_persist_grid<float>(h, s);
  }
  if (rc == CFR_OK) {
    unsigned *bar = h->p<unsigned>(h->b_bar);
    Barrier b;
    b.count = bar;
    b.gen = bar + 1;
    b.err = h->p<int>(h->b_err);
    b.spin_limit = h->opt.barrier_spin_limit > 0 ? h->opt.barrier_spin_limit : (int64_t)20000000;
    b.expected = (unsigned)h->persist_grid;
    int n_sync = (int)(2 * c.D * halves);
    long long iters = (long long)n;
    void *args[] = {&b, &n_sync, &iters};
    e = cudaMemsetAsync(bar, 0, 4, s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess)
      e = cudaLaunchCooperativeKernel((const void *)empty_persistent_kernel, dim3(h->persist_grid), dim3(kThreads), args, 0, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, b.err, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = set_err(CFR_ERR_DEVICE, "cfr_launch_floor: %s", cudaGetErrorString(e));
    else if (err) {
      cudaMemset(b.err, 0, 4);
      rc = set_err(CFR_ERR_TIMEOUT, "cfr_launch_floor: a grid barrier gave up waiting");
    } else {
      *persistent_ms = (double)ms / (double)n;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

extern "C" int cfr_autotune(cfr_handle *h, int reps, void *stream) {
  if (!h) return set_err(CFR_ERR_ARG, "cfr_autotune: null handle");
  if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "cfr_autotune: call cfr_bind first");
  if (reps < 1 || reps > 1000) return set_err(CFR_ERR_ARG, "cfr_autotune: reps must be in [1, 1000]");
  const Compiled &c = h->c;
  if (c.D == 0) return CFR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  // per-level candidates (kThreads = one set per block); the persistent kernel takes groups of at most a warp
  std::vector<int> cand = h->maxa_tier <= 8 ? std::vector<int>{1, 2, 4, 8, 16, 32, kThreads} : std::vector<int>{4, 8, 16, 32};
  std::vector<int> cand_p = h->maxa_tier <= 8 ? std::vector<int>{1, 2, 4, 8, 16, 32} : std::vector<int>{4, 8, 16, 32};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = CFR_OK;
  auto run_iter = [&]() -> int {
    return h->precision == CFR_P64 ? enqueue_iteration<double>(h, s) : enqueue_iteration<float>(h, s);
  };
  rc = run_iter();  // realistic reach and values for the trials
  for (int64_t d = c.D - 1; d >= 0 && rc == CFR_OK; --d) {
    int best = h->level_lanes[d];
    float best_ms = 1e30f;
    std::vector<int> cd = cand;
    // the streaming form works on one group of sets at a time with the whole
    // CTA: a candidate only where sets are long
    if (h->stream_ok[d] && c.level_mean_members[d] >= kStreamMinMembers) cd.push_back(kStreamLanes);
    for (int L : cd) {
      h->level_lanes[d] = L;
      rc = h->precision == CFR_P64 ? launch_bwd<double>(h, (int)d, s) : launch_bwd<float>(h, (int)d, s);
      if (rc) break;
      CK(cudaEventRecord(e0, s));
      for (int r = 0; r < reps && rc == CFR_OK; ++r)
        rc = h->precision == CFR_P64 ? launch_bwd<double>(h, (int)d, s) : launch_bwd<float>(h, (int)d, s);
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) { best_ms = ms; best = L; }
    }
    h->level_lanes[d] = best;
  }
  if (rc == CFR_OK && h->exec_form == CFR_EXEC_PERSISTENT) {
    int best = h->persist_lanes;
    float best_ms = 1e30f;
    for (int L : cand_p) {
      h->persist_lanes = L;
      h->persist_grid = 0;
      rc = h->precision == CFR_P64 ? launch_persistent_form<double>(h, 1, s) : launch_persistent_form<float>(h, 1, s);
      if (rc) break;
      CK(cudaEventRecord(e0, s));
      rc = h->precision == CFR_P64 ? launch_persistent_form<double>(h, reps, s) : launch_persistent_form<float>(h, reps, s);
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) { best_ms = ms; best = L; }
    }
    h->persist_lanes = best;
    h->persist_grid = 0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  drop_graphs(h);
  CK(cudaMemsetAsync(h->arena + h->b_err.off, 0, 16, s));
  if (c.n_wide) CK(cudaMemsetAsync(h->arena + h->b_wide_cnt.off, 0, 4 * c.n_wide, s));
  rc = h->precision == CFR_P64 ? init_state<double>(h, s) : init_state<float>(h, s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  return CFR_OK;
}

// ----------------------------------------------------------- batched solves
static int batch_table(cfr_handle *const *hs, int n, const int64_t *iters, int64_t n_iter, void *table_dev,
                       size_t table_bytes, int *maxa, int *precision, std::vector<InstDesc> &tab) {
  if (!hs || n <= 0) return set_err(CFR_ERR_ARG, "batch: no instances");
  if (!table_dev || table_bytes < sizeof(InstDesc) * (size_t)n)
    return set_err(CFR_ERR_ARG, "batch: the descriptor table needs %zu bytes", sizeof(InstDesc) * (size_t)n);
  if (reinterpret_cast<uintptr_t>(table_dev) % 16 != 0) return set_err(CFR_ERR_ARG, "batch: table must be 16-byte aligned");
  tab.resize(n);
  *maxa = 4;
  *precision = -1;
  for (int i = 0; i < n; ++i) {
    cfr_handle *h = hs[i];
    if (!h) return set_err(CFR_ERR_ARG, "batch: null handle %d", i);
    if (!h->bound) return set_err(CFR_ERR_NOT_BOUND, "batch: instance %d is not bound", i);
    if (*precision < 0) *precision = h->precision;
    else if (*precision != h->precision) return set_err(CFR_ERR_ARG, "batch: instances mix precisions");
    if (h->maxa_tier > 8) return set_err(CFR_ERR_UNSUPPORTED, "batch: instance %d has sets of more than 8 actions", i);
    *maxa = std::max(*maxa, h->maxa_tier);
    InstDesc &d = tab[i];
    memset(&d, 0, sizeof d);
    d.g = game_view(h);
    d.reach = h->arena + h->b_reach.off;
    d.v = h->arena + h->b_v.off;
    d.sigma = h->arena + h->b_sigma.off;
    d.R = h->p<double>(h->b_R);
    d.avg = h->p<double>(h->b_avg);
    d.t = h->p<long long>(h->b_t);
    d.lw = h->p<LevelWork>(h->b_levels);
    d.reach2 = h->p<double2>(h->b_reach2);
    d.vb = h->p<double2>(h->b_vb);
    d.vavg = h->p<double>(h->b_vavg);
    d.sbs = h->p<double>(h->b_sbs);
    d.out = h->p<double>(h->b_out);
    d.n_iter = iters ? iters[i] : n_iter;
    if (d.n_iter < 0) return set_err(CFR_ERR_ARG, "batch: negative iteration count");
    d.D = (int32_t)h->c.D;
    d.rule = h->rule;
    d.n_sets = (int32_t)h->c.I;
    d.root_vs = (int32_t)(h->c.N - 1);
    d.order = h->order;
  }
  return CFR_OK;
}

extern "C" size_t cfr_batch_table_bytes(int n) { return n > 0 ? sizeof(InstDesc) * (size_t)n : 0; }

extern "C" int cfr_batch_iterate(cfr_handle *const *hs, int n, const int64_t *iters, int64_t n_iter, void *table_dev,
                                 size_t table_bytes, int threads, int lanes, int cluster, void *stream) {
  std::vector<InstDesc> tab;
  int maxa = 4, prec = 0;
  int rc = batch_table(hs, n, iters, n_iter, table_dev, table_bytes, &maxa, &prec, tab);
  if (rc) return rc;
  if (threads == 0) threads = 256;
  if (lanes == 0) lanes = 4;
  if ((threads != 256 && threads != 1024) || (lanes != 2 && lanes != 4 && lanes != 8 && lanes != 32))
    return set_err(CFR_ERR_ARG, "batch: threads must be 256 or 1024 and lanes 2, 4, 8 or 32");
  if (cluster == 0) cluster = 1;
  if (cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8)
    return set_err(CFR_ERR_ARG, "batch: cluster must be 1, 2, 4 or 8 CTAs per instance");
  if (n == 0) return CFR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(table_dev, tab.data(), sizeof(InstDesc) * (size_t)n, cudaMemcpyHostToDevice, s));
  if (prec == CFR_P64) CK(launch_batch_iterate<double>(maxa, lanes, threads, cluster, n, s, (const InstDesc *)table_dev));
  else CK(launch_batch_iterate<float>(maxa, lanes, threads, cluster, n, s, (const InstDesc *)table_dev));
  for (int i = 0; i < n; ++i) hs[i]->iteration_host += tab[i].n_iter;
  return CFR_OK;
}

extern "C" int cfr_batch_exploitability(cfr_handle *const *hs, int n, double *out, void *table_dev, size_t table_bytes,
                                        int threads, int lanes, void *stream) {
  if (!out) return set_err(CFR_ERR_ARG, "batch: null output");
  std::vector<InstDesc> tab;
  int maxa = 4, prec = 0;
  int rc = batch_table(hs, n, nullptr, 0, table_dev, table_bytes, &maxa, &prec, tab);
  if (rc) return rc;
  if (threads == 0) threads = 256;
  if (lanes == 0) lanes = 4;
  if ((threads != 256 && threads != 1024) || (lanes != 2 && lanes != 4 && lanes != 8 && lanes != 32))
    return set_err(CFR_ERR_ARG, "batch: threads must be 256 or 1024 and lanes 2, 4, 8 or 32");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(table_dev, tab.data(), sizeof(InstDesc) * (size_t)n, cudaMemcpyHostToDevice, s));
  CK(launch_batch_br(maxa, lanes, threads, n, s, (const InstDesc *)table_dev));
  for (int i = 0; i < n; ++i) CK(cudaMemcpyAsync(out + 4 * i, tab[i].out, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return CFR_OK;
}
