// pond_batch.cu -- many contexts advanced together by the member step kernel
// on a persistent grid, one launch per time step (pond_batch_* of
// include/pond.h).
//
// A launch is one time step of every member that still has steps to take in
// the current chunk.  The members' tiles are numbered consecutively (member i
// owns tiles [tile_begin_i, tile_begin_i + tiles_i)); a grid of
// (SMs x resident CTAs) CTAs strides over all tiles, each tile running the
// same tile step as the single-context kernel, with the member's own
// constants, buffers and status block taken from a descriptor table in
// device memory.  The member count and the tile count are read from that
// table as well, so one captured CUDA graph of G launches serves every chunk
// while members join and leave; only the table (a few hundred bytes per
// member) is uploaded per chunk.
//
// A member's state is bit for bit the same alone (pond_step) and in any batch
// with the same tile shape: both launch the same kernel function, and every
// output depends only on its stencil's arithmetic.  Every shape computes the
// same step (to rounding, as separate machine code), which lets the
// autotuner time candidate shapes on real steps: the steps it times are
// steps of the run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "pond_internal.h"

using pond::State;
using pond::StepConst;
using pond::Stats;
using pond_detail::state_of;

using pond::InstDesc;
using pond::Shape;
using pond::TableHdr;

namespace {

// candidate shapes of a batch, the default first (tile codes of pond_params.tile)
std::vector<Shape> batch_shapes(bool fp32, int D) {
  const std::vector<Shape> all = fp32 ? pond_shapes_fp32(D) : pond_shapes_fp64(D);
  if (D == 1) return all;
  static const int kMixed[3] = {10, 11, 6}, kFp64[3] = {10, 9, 6};
  const int *codes = fp32 ? kMixed : kFp64;
  std::vector<Shape> out;
  for (int i = 0; i < 3; ++i)
    for (const Shape &s : all)
      if (s.code == codes[i]) out.push_back(s);
  return out;
}

}  // namespace

struct pond_batch {
  int D;
  bool fp32;
  cudaStream_t stream;
  int capacity;
  pond_tune tune;
  std::vector<pond_ctx *> members;
  std::vector<Shape> shapes;
  std::vector<int> occupancy;  // CTAs per SM of each shape
  int shape;                   // index of the shape in use
  int grid;
  int sms;
  bool tuned;
  bool autotuning;             // the autotuner picks the shape (tile 0, autotune on)
  long long tuned_tiles;       // tiles (first candidate's shape) the shape was tuned on
  double tuned_mlups;
  unsigned char *dtable;
  size_t desc_bytes, table_bytes;
  unsigned char *htable[2];
  cudaEvent_t hdone[2];
  int hslot;
  cudaGraphExec_t graph;
  int graph_shape;
};

namespace {

size_t desc_size(bool fp32) { return fp32 ? sizeof(InstDesc<float>) : sizeof(InstDesc<double>); }

int tiles_x_of(const pond_ctx *c, const Shape &s) { return (int)((c->nx + s.bx - 1) / s.bx); }
int tiles_y_of(const pond_ctx *c, const Shape &s) {
  return c->D == 2 ? (int)((c->ny + s.by - 1) / s.by) : 1;
}
int tiles_of(const pond_ctx *c, const Shape &s) { return tiles_x_of(c, s) * tiles_y_of(c, s); }

template <typename R>
void fill_desc(unsigned char *dst, const pond_ctx *c, const Shape &s, int tile_begin, int steps) {
  InstDesc<R> d;
  memset(&d, 0, sizeof(d));
  d.K = c->K;
  d.S[0] = state_of<R>(c, 0);
  d.S[1] = state_of<R>(c, 1);
  d.stats = c->stats;
  d.tiles_x = tiles_x_of(c, s);
  d.tile_begin = tile_begin;
  d.steps = steps;
  d.parity = c->cur;
  memcpy(dst, &d, sizeof(d));
}

// uploads the table of the members with steps[i] > 0 for shape s; returns the
// number of cells in it
pond_status upload_table(pond_batch *b, int shape, const std::vector<int> &steps, size_t *cells) {
  const Shape &s = b->shapes[shape];
  const int slot = b->hslot;
  b->hslot ^= 1;
  // the pinned buffer may still be read by the copy queued two chunks ago
  POND_CUDA(cudaEventSynchronize(b->hdone[slot]));
  unsigned char *h = b->htable[slot];
  TableHdr hdr;
  memset(&hdr, 0, sizeof(hdr));
  // strips of two tiles where the grid still strides over at least four
  // strips per CTA (members with different step counts drop out of later
  // launches, and many small units keep the CTAs balanced), else single tiles
  const int slots = b->sms * std::max(1, b->occupancy[shape]);
  long long all_tiles = 0;
  for (size_t i = 0; i < b->members.size(); ++i)
    if (steps[i] > 0) all_tiles += tiles_of(b->members[i], s);
  int strip = 1;
  while (strip < pond::kMaxAutoStrip && all_tiles / (2 * strip) >= 4LL * slots) strip *= 2;
  size_t ncell = 0;
  int unit = 0;
  for (size_t i = 0; i < b->members.size(); ++i) {
    if (steps[i] <= 0) continue;
    const pond_ctx *c = b->members[i];
    unsigned char *dst = h + sizeof(TableHdr) + (size_t)hdr.n * b->desc_bytes;
    if (b->fp32) fill_desc<float>(dst, c, s, unit, steps[i]);
    else fill_desc<double>(dst, c, s, unit, steps[i]);
    unit += pond::strips_of(tiles_x_of(c, s), tiles_y_of(c, s), strip);
    ncell += (size_t)c->N;
    ++hdr.n;
  }
  hdr.total_tiles = unit;
  hdr.strip = strip;
  memcpy(h, &hdr, sizeof(hdr));
  POND_CUDA(cudaMemcpyAsync(b->dtable, h, sizeof(TableHdr) + (size_t)hdr.n * b->desc_bytes,
                            cudaMemcpyHostToDevice, b->stream));
  POND_CUDA(cudaEventRecord(b->hdone[slot], b->stream));
  *cells = ncell;
  return POND_OK;
}

pond_status launch_chunk(pond_batch *b, int shape, int launches, bool use_graph) {
  const Shape &s = b->shapes[shape];
  const int grid = b->sms * std::max(1, b->occupancy[shape]);
  if (use_graph && launches == b->tune.graph_steps && b->stream) {
    if (!b->graph || b->graph_shape != shape) {
      if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
      cudaGraph_t g = nullptr;
      POND_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      for (int k = 0; k < launches; ++k) s.launch(b->dtable, k, grid, b->stream);
      cudaError_t e = cudaStreamEndCapture(b->stream, &g);
      if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        return POND_E_CUDA;
      }
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { (void)cudaGetLastError(); b->graph = nullptr; return POND_E_CUDA; }
      b->graph_shape = shape;
    }
    POND_CUDA(cudaGraphLaunch(b->graph, b->stream));
    return POND_OK;
  }
  for (int k = 0; k < launches; ++k) s.launch(b->dtable, k, grid, b->stream);
  POND_CUDA(cudaGetLastError());
  return POND_OK;
}

// advances member i by steps[i] (<= G) in one chunk with shape `shape`
pond_status run_chunk(pond_batch *b, int shape, std::vector<int> &steps, bool use_graph,
                      size_t *cells, int *launches) {
  int mx = 0;
  for (int s : steps) mx = std::max(mx, s);
  *launches = mx;
  *cells = 0;
  if (mx == 0) return POND_OK;
  pond_status st = upload_table(b, shape, steps, cells);
  if (st != POND_OK) return st;
  if ((st = launch_chunk(b, shape, mx, use_graph)) != POND_OK) return st;
  for (size_t i = 0; i < b->members.size(); ++i) {
    pond_ctx *c = b->members[i];
    c->cur ^= steps[i] & 1;
    c->steps += steps[i];
  }
  return POND_OK;
}

}  // namespace

// called by pond_destroy(): a destroyed context leaves its batch
void pond_batch_detach(pond_ctx *c) {
  if (!c || !c->batch) return;
  pond_batch *b = static_cast<pond_batch *>(c->batch);
  b->members.erase(std::remove(b->members.begin(), b->members.end(), c), b->members.end());
  c->batch = nullptr;
}

extern "C" {

void pond_tune_default(pond_tune *t) {
  if (!t) return;
  memset(t, 0, sizeof(*t));
  t->tile = 0;
  t->graph_steps = 8;
  t->autotune = 1;
}

pond_status pond_batch_create(pond_batch **out, int32_t dim, int32_t precision, int32_t capacity,
                              const pond_tune *tune, void *stream) {
  if (!out) return POND_E_INVAL;
  *out = nullptr;
  if ((dim != 1 && dim != 2) || (precision != POND_FP64 && precision != POND_FP32_MIXED) ||
      capacity < 1 || capacity > (1 << 20))
    return POND_E_INVAL;
  pond_tune t;
  pond_tune_default(&t);
  if (tune) t = *tune;
  if (t.graph_steps < 1 || t.graph_steps > 1024) return POND_E_INVAL;
  pond_batch *b = new (std::nothrow) pond_batch();
  if (!b) return POND_E_NOMEM;
  b->D = dim;
  b->fp32 = precision == POND_FP32_MIXED;
  b->stream = (cudaStream_t)stream;
  b->capacity = capacity;
  b->tune = t;
  b->shapes = batch_shapes(b->fp32, dim);
  if (b->shapes.empty()) {
    delete b;
    return POND_E_INVAL;
  }
  b->shape = 0;
  if (t.tile) {
    b->shape = -1;
    for (size_t i = 0; i < b->shapes.size(); ++i)
      if (b->shapes[i].code == t.tile) b->shape = (int)i;
    if (b->shape < 0) { delete b; return POND_E_INVAL; }
  }
  b->tuned = t.tile != 0 || !t.autotune || b->shapes.size() == 1;
  b->autotuning = !b->tuned;
  b->tuned_tiles = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    delete b;
    return POND_E_CUDA;
  }
  for (const Shape &s : b->shapes) {
    int occ = 0;
    if (s.prepare(&occ) != cudaSuccess) { (void)cudaGetLastError(); delete b; return POND_E_CUDA; }
    b->occupancy.push_back(occ);
  }
  b->desc_bytes = desc_size(b->fp32);
  b->table_bytes = sizeof(TableHdr) + (size_t)capacity * b->desc_bytes;
  bool ok = cudaMalloc((void **)&b->dtable, b->table_bytes) == cudaSuccess;
  for (int i = 0; i < 2 && ok; ++i) {
    ok = cudaMallocHost((void **)&b->htable[i], b->table_bytes) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->hdone[i], cudaEventDisableTiming) == cudaSuccess;
    if (ok) ok = cudaEventRecord(b->hdone[i], b->stream) == cudaSuccess;
  }
  if (!ok) {
    (void)cudaGetLastError();
    pond_batch_destroy(b);
    return POND_E_NOMEM;
  }
  *out = b;
  return POND_OK;
}

void pond_batch_destroy(pond_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  for (pond_ctx *c : b->members) c->batch = nullptr;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->dtable) cudaFree(b->dtable);
  for (int i = 0; i < 2; ++i) {
    if (b->htable[i]) cudaFreeHost(b->htable[i]);
    if (b->hdone[i]) cudaEventDestroy(b->hdone[i]);
  }
  (void)cudaGetLastError();
  delete b;
}

pond_status pond_batch_add(pond_batch *b, pond_ctx *c) {
  if (!b || !c) return POND_E_INVAL;
  if (!c->inited) return POND_E_STATE;
  if (c->batch || c->D != b->D || c->qf1 != 4 || c->qg1 != 3 || c->K.ms || c->fp32 != b->fp32 || c->stream != b->stream ||
      c->K.iterative || (int)b->members.size() >= b->capacity)
    return POND_E_INVAL;
  b->members.push_back(c);
  c->batch = b;
  return POND_OK;
}

pond_status pond_batch_remove(pond_batch *b, pond_ctx *c) {
  if (!b || !c || c->batch != b) return POND_E_INVAL;
  pond_batch_detach(c);
  return POND_OK;
}

int32_t pond_batch_size(const pond_batch *b) { return b ? (int32_t)b->members.size() : 0; }

pond_status pond_batch_step(pond_batch *b, const int64_t *steps) {
  if (!b) return POND_E_INVAL;
  const size_t n = b->members.size();
  std::vector<int64_t> left(n);
  for (size_t i = 0; i < n; ++i) {
    left[i] = steps ? steps[i] : 1;
    if (left[i] < 0) return POND_E_INVAL;
    if (!b->members[i]->inited) return POND_E_STATE;
  }
  const int G = b->tune.graph_steps;
  std::vector<int> chunk(n);
  auto next_chunk = [&]() {
    int64_t mx = 0;
    for (size_t i = 0; i < n; ++i) {
      chunk[i] = (int)std::min<int64_t>(left[i], G);
      mx = std::max<int64_t>(mx, left[i]);
    }
    return mx;
  };
  pond_status st;
  size_t cells;
  int launches;
  // autotune: one full chunk per candidate shape, on real steps (every shape
  // gives the same result), timed with events; then the fastest is kept until
  // the batch's work (its stepping members' tiles) has grown or shrunk
  // fourfold since, when the shapes are timed again (a serving batch is often
  // tuned on its first, small member)
  long long cur_tiles = 0;
  for (size_t i = 0; i < n; ++i)
    if (left[i] > 0) cur_tiles += tiles_of(b->members[i], b->shapes[0]);
  if (b->autotuning && b->tuned && cur_tiles > 0 &&
      (cur_tiles > 4 * b->tuned_tiles || 4 * cur_tiles < b->tuned_tiles))
    b->tuned = false;
  if (!b->tuned) {
    int64_t mn = INT64_MAX;
    for (size_t i = 0; i < n; ++i) mn = std::min(mn, left[i]);
    if (n > 0 && mn >= (int64_t)G * (int64_t)b->shapes.size()) {
      std::vector<cudaEvent_t> ev(2 * b->shapes.size(), nullptr);
      std::vector<size_t> cell(b->shapes.size());
      for (auto &e : ev) POND_CUDA(cudaEventCreate(&e));
      for (size_t s = 0; s < b->shapes.size(); ++s) {
        next_chunk();
        POND_CUDA(cudaEventRecord(ev[2 * s], b->stream));
        if ((st = run_chunk(b, (int)s, chunk, false, &cell[s], &launches)) != POND_OK) return st;
        POND_CUDA(cudaEventRecord(ev[2 * s + 1], b->stream));
        for (size_t i = 0; i < n; ++i) left[i] -= chunk[i];
      }
      POND_CUDA(cudaEventSynchronize(ev.back()));
      double best = 0.0;
      for (size_t s = 0; s < b->shapes.size(); ++s) {
        float ms = 0.f;
        POND_CUDA(cudaEventElapsedTime(&ms, ev[2 * s], ev[2 * s + 1]));
        const double mlups = ms > 0.f ? (double)cell[s] * G / (ms * 1e-3) / 1e6 : 0.0;
        if (mlups > best) { best = mlups; b->shape = (int)s; }
      }
      for (auto &e : ev) cudaEventDestroy(e);
      b->tuned = true;
      b->tuned_tiles = cur_tiles;
      b->tuned_mlups = best;
    }
  }
  while (next_chunk() > 0) {
    if ((st = run_chunk(b, b->shape, chunk, true, &cells, &launches)) != POND_OK) return st;
    for (size_t i = 0; i < n; ++i) left[i] -= chunk[i];
  }
  return POND_OK;
}

pond_status pond_batch_info(const pond_batch *b, int32_t *tile, int32_t *grid, int32_t *tuned,
                            double *tuned_mlups) {
  if (!b) return POND_E_INVAL;
  if (tile) *tile = b->shapes[b->shape].code;
  if (grid) *grid = b->sms * std::max(1, b->occupancy[b->shape]);
  if (tuned) *tuned = b->tuned ? 1 : 0;
  if (tuned_mlups) *tuned_mlups = b->tuned_mlups;
  return POND_OK;
}

}  // extern "C"
