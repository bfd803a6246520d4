// Batched reconstruction of many independent slices of uneven size and view count.
//
// Per distinct geometry (N, views, detector, blur) the batch builds one Gram filter
// (taps, spectrum, twiddles) and one set of back-projection tables; every slice gets
// its own CG state (scratch, r, p, q, scalars) that points at its geometry's shared
// spectrum.  bsct_batch_solve records, for every slice, prefilter + back projection +
// CG start + n CG iterations as one branch of a CUDA graph (the slices are spread over
// a pool of streams forked from and joined back to the caller's stream), instantiates
// the graph once and replays it with a single launch; the graph is re-recorded only
// when the sinogram / output pointers or the iteration count change.
#include <string.h>

#include <vector>

#include "bsct_internal.h"

namespace {

struct BatchGeom {
  bsct_geom g{};
  std::vector<double> angles;
  bsct_gram* filt = nullptr;
  bsct::BpPlan bp;
};

struct BatchSlice {
  int geom = 0;
  bsct_gram* st = nullptr;  // CG state sharing the geometry's filter
  float* ct = nullptr;      // prefiltered sinogram [views][bins]
  float* b = nullptr;       // right-hand side [N][N]
};

bool same_geom(const bsct_geom& a, const bsct_geom& b) {
  if (a.N != b.N || a.n_angles != b.n_angles || a.n_bins != b.n_bins || a.lambda_y != b.lambda_y ||
      a.zeta_blur != b.zeta_blur)
    return false;
  return memcmp(a.angles_pi, b.angles_pi, sizeof(double) * a.n_angles) == 0;
}

}  // namespace

struct bsct_batch {
  std::vector<BatchGeom> geoms;
  std::vector<BatchSlice> slices;
  std::vector<cudaStream_t> pool;
  std::vector<float*> pool_part;  // per pool stream: back-projection partial images of its slices
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;  // non-blocking stream the graph is recorded on
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> bound_sino;
  std::vector<void*> bound_x;
  int bound_iters = -1;
  unsigned long long kernels_per_launch = 0;
  size_t graph_nodes = 0;
};

static void batch_release(bsct_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto& s : b->slices) {
    bsct_gram_free(s.st);
    cudaFree(s.ct);
    cudaFree(s.b);
  }
  for (auto& g : b->geoms) {
    bsct_gram_free(g.filt);
    cudaFree(g.bp.ang);
    cudaFree(g.bp.p00);
    cudaFree(g.bp.csl);
    cudaFree(g.bp.tab);
    cudaFree(g.bp.status);
  }
  for (auto s : b->pool) cudaStreamDestroy(s);
  for (auto q : b->pool_part) cudaFree(q);
  for (auto e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

extern "C" void bsct_batch_free(bsct_batch* b) { batch_release(b); }

#define BTRY(expr)                                              \
  do {                                                          \
    int _rc = (expr);                                           \
    if (_rc != BSCT_OK) { batch_release(bt); return _rc; }      \
  } while (0)
#define BCTRY(expr)                                                                             \
  do {                                                                                          \
    cudaError_t _e = (expr);                                                                    \
    if (_e != cudaSuccess) { bsct_set_last_cuda_error(_e); batch_release(bt); return BSCT_ERR_CUDA; } \
  } while (0)

extern "C" int bsct_batch_create(int n_slices, const bsct_geom* geoms, bsct_batch** out, void* stream) {
  using namespace bsct;
  if (n_slices < 1 || !geoms || !out) {
    bsct_set_last_message("invalid argument");
    return BSCT_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n_slices; ++i) {
    int rc = bsct_check_geom(&geoms[i]);
    if (rc == BSCT_OK) rc = bsct_check_bp_geom(&geoms[i]);
    if (rc != BSCT_OK) return rc;
    if (!bsct_supported_size(geoms[i].N)) {
      bsct_set_last_message("unsupported N in batch");
      return BSCT_ERR_UNSUPPORTED_SIZE;
    }
    double w[2];
    if (bsct_blur_boxes(&geoms[i], w) == 2) {
      bsct_set_last_message("batch: two detector boxes are not supported (the back projection tables hold one)");
      return BSCT_ERR_UNSUPPORTED_SIZE;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  bsct_batch* bt = new bsct_batch();
  bt->slices.resize(n_slices);
  for (int i = 0; i < n_slices; ++i) {
    // a one-entry box list is the single detector box zeta_blur
    bsct_geom gi_geom = geoms[i];
    double w[2];
    gi_geom.zeta_blur = bsct_blur_boxes(&geoms[i], w) == 1 ? w[0] : 0.0;
    gi_geom.n_blur = 0;
    gi_geom.blur_widths = nullptr;
    int gi = -1;
    for (size_t k = 0; k < bt->geoms.size(); ++k)
      if (same_geom(bt->geoms[k].g, gi_geom)) { gi = (int)k; break; }
    if (gi < 0) {
      bt->geoms.emplace_back();
      BatchGeom& G = bt->geoms.back();
      G.g = gi_geom;
      G.angles.assign(geoms[i].angles_pi, geoms[i].angles_pi + geoms[i].n_angles);
      G.g.angles_pi = G.angles.data();
      gi = (int)bt->geoms.size() - 1;
    }
    bt->slices[i].geom = gi;
  }
  // per geometry: Gram filter and back-projection tables
  for (auto& G : bt->geoms) {
    BTRY(bsct_gram_build(&G.g, BSCT_F32, &G.filt, stream));
    BpPlan& p = G.bp;
    p.N = G.g.N; p.na = G.g.n_angles; p.M = G.g.n_bins; p.lambda = G.g.lambda_y; p.zeta = G.g.zeta_blur;
    BCTRY(cudaMalloc(&p.ang, p.na * sizeof(double)));
    BCTRY(cudaMalloc(&p.p00, p.na * sizeof(double)));
    BCTRY(cudaMalloc(&p.csl, p.na * sizeof(double2)));
    BCTRY(cudaMalloc(&p.tab, bp_table_bytes(p.na, BSCT_F32)));
    BCTRY(cudaMalloc(&p.status, sizeof(int)));
    BCTRY(cudaMemcpyAsync(p.ang, G.angles.data(), p.na * sizeof(double), cudaMemcpyHostToDevice, st));
    BTRY(bp_make_tables<float>(p, st));
  }
  // per slice: CG state sharing the filter, prefilter scratch, right-hand side
  for (auto& S : bt->slices) {
    const BatchGeom& G = bt->geoms[S.geom];
    const int N = G.g.N;
    bsct_gram* c = new bsct_gram();
    c->owns_filter = false;
    c->N = N; c->precision = BSCT_F32; c->n_angles = G.filt->n_angles;
    c->zeta = G.filt->zeta; c->lambda = G.filt->lambda;
    c->taps = G.filt->taps; c->Gt64 = G.filt->Gt64; c->Gt32 = G.filt->Gt32; c->tw = G.filt->tw;
    S.st = c;
    BCTRY(cudaMalloc(&c->S, (size_t)N * N * 2 * sizeof(float)));
    BCTRY(cudaMalloc(&c->r, (size_t)N * N * sizeof(float)));
    BCTRY(cudaMalloc(&c->p, (size_t)N * N * sizeof(float)));
    BCTRY(cudaMalloc(&c->q, (size_t)N * N * sizeof(float)));
    c->n_partials = 1024;
    BCTRY(cudaMalloc(&c->partials, (size_t)c->n_partials * 2 * sizeof(double)));
    BCTRY(cudaMalloc(&c->scal, 16 * sizeof(double)));
    BCTRY(cudaMemsetAsync(c->scal, 0, 16 * sizeof(double), st));
    BCTRY(cudaMalloc(&S.ct, (size_t)G.g.n_angles * G.g.n_bins * sizeof(float)));
    BCTRY(cudaMalloc(&S.b, (size_t)N * N * sizeof(float)));
  }
  // one eager apply / CG step per size outside any capture (one-time kernel attributes)
  std::vector<int> seen;
  for (auto& S : bt->slices) {
    const int N = S.st->N;
    bool done = false;
    for (int n : seen) done |= (n == N);
    if (done) continue;
    seen.push_back(N);
    BCTRY(cudaMemsetAsync(S.b, 0, (size_t)N * N * sizeof(float), st));
    BTRY(bsct_cg_begin(S.st, S.b, S.st->q, 1, stream));
    BTRY(bsct_cg_iterate(S.st, S.st->q, 1, stream));
  }
  const int npool = n_slices < 32 ? n_slices : 32;
  bt->pool.resize(npool);
  bt->joins.resize(npool);
  bt->pool_part.assign(npool, nullptr);
  for (int k = 0; k < npool; ++k) {  // slices i with i % npool == k run in order on stream k
    size_t need = 0;
    for (size_t i = k; i < bt->slices.size(); i += npool) {
      const bsct_geom& g = bt->geoms[bt->slices[i].geom].g;
      const size_t nb = bp_partial_bytes(g.N, g.n_angles, g.lambda_y, BSCT_F32);
      need = nb > need ? nb : need;
    }
    if (need) BCTRY(cudaMalloc(&bt->pool_part[k], need));
  }
  for (int k = 0; k < npool; ++k) {
    BCTRY(cudaStreamCreateWithFlags(&bt->pool[k], cudaStreamNonBlocking));
    BCTRY(cudaEventCreateWithFlags(&bt->joins[k], cudaEventDisableTiming));
  }
  BCTRY(cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming));
  BCTRY(cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking));
  BCTRY(cudaStreamSynchronize(st));
  *out = bt;
  return BSCT_OK;
}
#undef BTRY
#undef BCTRY

// records on the batch's own non-blocking stream (the caller's stream may be the legacy
// default stream, which cannot be captured); the graph is launched on the caller's stream
static int batch_record(bsct_batch* bt, const float* const* sino, float* const* x, int iters) {
  using namespace bsct;
  cudaStream_t st = bt->cap;
  cudaGraph_t graph = nullptr;
  const unsigned long long k0 = bsct_launch_count();
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { bsct_set_last_cuda_error(e); return BSCT_ERR_CUDA; }
  int rc = BSCT_OK;
  e = cudaEventRecord(bt->fork, st);
  for (size_t k = 0; e == cudaSuccess && k < bt->pool.size(); ++k) e = cudaStreamWaitEvent(bt->pool[k], bt->fork, 0);
  for (size_t i = 0; e == cudaSuccess && rc == BSCT_OK && i < bt->slices.size(); ++i) {
    BatchSlice& S = bt->slices[i];
    cudaStream_t s = bt->pool[i % bt->pool.size()];
    BpPlan bp = bt->geoms[S.geom].bp;
    bp.part = bt->pool_part[i % bt->pool.size()];
    rc = bp_apply<float>(bp, sino[i], S.ct, S.b, s);
    if (rc == BSCT_OK) rc = bsct_cg_begin(S.st, S.b, x[i], 1, s);
    if (rc == BSCT_OK && iters > 0) rc = bsct_cg_iterate(S.st, x[i], iters, s);
  }
  for (size_t k = 0; e == cudaSuccess && k < bt->pool.size(); ++k) {
    e = cudaEventRecord(bt->joins[k], bt->pool[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, bt->joins[k], 0);
  }
  cudaError_t e2 = cudaStreamEndCapture(st, &graph);
  if (e == cudaSuccess) e = e2;
  if (rc != BSCT_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (rc == BSCT_OK) { bsct_set_last_cuda_error(e); rc = BSCT_ERR_CUDA; }
    return rc;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    bsct_set_last_cuda_error(e);
    return BSCT_ERR_CUDA;
  }
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  bt->graph = graph;
  bt->exec = exec;
  bt->kernels_per_launch = bsct_launch_count() - k0;
  bsct::g_launches.fetch_sub(bt->kernels_per_launch);  // recorded, not launched
  size_t nn = 0;
  cudaGraphGetNodes(graph, nullptr, &nn);
  bt->graph_nodes = nn;
  bt->bound_sino.assign(sino, sino + bt->slices.size());
  bt->bound_x.assign(x, x + bt->slices.size());
  bt->bound_iters = iters;
  return BSCT_OK;
}

extern "C" int bsct_batch_solve(bsct_batch* bt, const float* const* d_sino, float* const* d_x, int cg_iters,
                                void* stream) {
  if (!bt || !d_sino || !d_x || cg_iters < 0) {
    bsct_set_last_message("invalid argument");
    return BSCT_ERR_INVALID_ARG;
  }
  for (size_t i = 0; i < bt->slices.size(); ++i)
    if (!d_sino[i] || !d_x[i]) {
      bsct_set_last_message("NULL slice pointer");
      return BSCT_ERR_INVALID_ARG;
    }
  cudaStream_t st = (cudaStream_t)stream;
  bool same = bt->exec && bt->bound_iters == cg_iters;
  for (size_t i = 0; same && i < bt->slices.size(); ++i)
    same = bt->bound_sino[i] == (const void*)d_sino[i] && bt->bound_x[i] == (void*)d_x[i];
  if (!same) {
    const int rc = batch_record(bt, d_sino, d_x, cg_iters);
    if (rc != BSCT_OK) return rc;
  }
  BSCT_CUDA_TRY(cudaGraphLaunch(bt->exec, st));
  bsct::g_launches.fetch_add(bt->kernels_per_launch);
  return BSCT_OK;
}

extern "C" int bsct_batch_info(const bsct_batch* bt, int* n_geometries, long long* graph_nodes,
                               long long* kernels_per_launch) {
  if (!bt) {
    bsct_set_last_message("NULL batch");
    return BSCT_ERR_INVALID_ARG;
  }
  if (n_geometries) *n_geometries = (int)bt->geoms.size();
  if (graph_nodes) *graph_nodes = (long long)bt->graph_nodes;
  if (kernels_per_launch) *kernels_per_launch = (long long)bt->kernels_per_launch;
  return BSCT_OK;
}
