// C ABI of libsp2.so (declared in include/sp2.h) and the host-side drivers of
// the SP2 recursions. The host only sequences kernels on the handle's stream;
// every arithmetic step (bounds, scaling, products, branch choice, stopping
// test, response updates, contractions) runs on the device.
#include <stdarg.h>
#include <algorithm>
#include <cmath>
#include <stdio.h>
#include <string.h>

#include <map>
#include <string>
#include <vector>

#include "sp2_internal.h"

using namespace sp2;

struct sp2_handle_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t limit = 0;
  size_t held = 0;
  std::string err;
  struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
  };
  std::map<std::string, Buf> bufs;
  struct TileList {
    Tile* d = nullptr;
    int n = 0;
  };
  std::map<std::string, TileList> tiles;
  DevState* d_state = nullptr;
  DevState* h_state = nullptr;  // pinned mirror
  TcTuning tune;                // product-kernel launch settings (sp2_set_option)
  // The step loop reads the trailing part of the device state after every step
  // into a pinned ring (kRing slots), each followed by an event; the host waits
  // only for the step kLookahead behind the one it enqueues, so the GPU never
  // idles and at most kLookahead no-op steps follow the stop.
  static constexpr int kRing = 16, kLookahead = 8;
  DevState* ring = nullptr;     // pinned, kRing snapshots (tail only)
  cudaEvent_t ring_ev[kRing] = {};
  // side stream for host copies that overlap later work of the same call
  cudaStream_t side = nullptr;
  cudaEvent_t side_ev[2] = {};
  bool side_pending = false;
  std::vector<cudaEvent_t> events;  // pool for time_kernels (start/stop pairs)

  // X_n history kept for sp2_adjoint
  struct History {
    bool valid = false;
    int64_t n = 0, np = 0;
    int mode = 0, M = 0, k = 4;
    int tail = 0;            // split-tail mode of the kept recursion
    double beta = 0.0;
    std::vector<int> sigma;  // sigma[1..M] (filled when the producing call completes)
  } hist;

  // the work of the last call that has not been waited for (sp2_synchronize)
  struct Pending;
  Pending* pending = nullptr;
};

namespace {

int fail(sp2_handle_t h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  return code;
}

#define CK(expr)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(h, SP2_ECUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                   \
  } while (0)

#define TRY(expr)            \
  do {                       \
    int r_ = (expr);         \
    if (r_ != SP2_OK) return r_; \
  } while (0)

// --------------------------------------------------------------- workspace
int ws(sp2_handle_t h, const std::string& name, size_t bytes, void** out) {
  if (bytes == 0) bytes = 256;
  auto& b = h->bufs[name];
  if (b.bytes >= bytes) {
    *out = b.p;
    return SP2_OK;
  }
  if (b.p) {
    cudaFree(b.p);
    h->held -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
  }
  if (h->limit && h->held + bytes > h->limit)
    return fail(h, SP2_ENOMEM, "workspace limit %zu bytes exceeded (need %zu more for %s)",
                h->limit, bytes, name.c_str());
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, SP2_ENOMEM, "cudaMalloc(%zu) for %s failed: %s", bytes, name.c_str(),
                cudaGetErrorString(e));
  }
  b.p = p;
  b.bytes = bytes;
  h->held += bytes;
  *out = p;
  return SP2_OK;
}

void ws_free(sp2_handle_t h, const std::string& name) {
  auto it = h->bufs.find(name);
  if (it == h->bufs.end()) return;
  if (it->second.p) {
    cudaFree(it->second.p);
    h->held -= it->second.bytes;
  }
  h->bufs.erase(it);
}

size_t master_size(int mode) { return mode == SP2_MODE_FP64 ? 8 : 4; }

int mat(sp2_handle_t h, const std::string& name, int64_t rows, int64_t np, int mode, MatBuf* m) {
  const size_t cnt = (size_t)rows * (size_t)np;
  *m = MatBuf{};
  TRY(ws(h, name + ".m", cnt * master_size(mode), &m->master));
  if (split_mode(mode)) {
    void* p;
    TRY(ws(h, name + ".h", cnt * 2, &p));
    m->hi = static_cast<uint16_t*>(p);
    TRY(ws(h, name + ".l", cnt * 2, &p));
    m->lo = static_cast<uint16_t*>(p);
    if (n_planes(mode) == 3) {
      TRY(ws(h, name + ".d", cnt * 2, &p));
      m->mid = static_cast<uint16_t*>(p);
    }
  }
  return SP2_OK;
}

// FP16X2 per-matrix scale state for a batch of B response matrices
int scales(sp2_handle_t h, const std::string& name, int64_t B, ScaleBuf* sc) {
  void* p;
  TRY(ws(h, name, (size_t)B * 5 * sizeof(float), &p));
  float* f = static_cast<float*>(p);
  sc->ymax = f;
  sc->yscale = f + 2 * B;
  sc->zmax = f + 4 * B;
  sc->B = B;
  return SP2_OK;
}

// --------------------------------------------------------------- host/device staging
bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int stage_in(sp2_handle_t h, const std::string& name, const void* p, size_t bytes,
             const void** dev) {
  if (bytes == 0 || is_device_ptr(p)) {
    *dev = p;
    return SP2_OK;
  }
  void* d;
  TRY(ws(h, "stage." + name, bytes, &d));
  CK(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, h->stream));
  *dev = d;
  return SP2_OK;
}

struct OutStage {
  void* user = nullptr;
  void* dev = nullptr;
  size_t bytes = 0;
  bool host = false;
};

int stage_out(sp2_handle_t h, const std::string& name, void* p, size_t bytes, OutStage* o) {
  o->user = p;
  o->bytes = bytes;
  o->host = !(bytes == 0 || is_device_ptr(p));
  if (!o->host) {
    o->dev = p;
    return SP2_OK;
  }
  return ws(h, "stage." + name, bytes, &o->dev);
}

int finish_out(sp2_handle_t h, const OutStage& o) {
  if (o.host) CK(cudaMemcpyAsync(o.user, o.dev, o.bytes, cudaMemcpyDeviceToHost, h->stream));
  return SP2_OK;
}

// The host copy of an output that is final while later work of the call still
// runs: on the handle's side stream, after what the main stream has enqueued so
// far; join_beside makes the main stream wait for it.
int finish_out_beside(sp2_handle_t h, const OutStage& o) {
  if (!o.host) return SP2_OK;
  if (!h->side) {
    CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->side_ev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->side_ev[1], cudaEventDisableTiming));
  }
  CK(cudaEventRecord(h->side_ev[0], h->stream));
  CK(cudaStreamWaitEvent(h->side, h->side_ev[0], 0));
  CK(cudaMemcpyAsync(o.user, o.dev, o.bytes, cudaMemcpyDeviceToHost, h->side));
  CK(cudaEventRecord(h->side_ev[1], h->side));
  h->side_pending = true;
  return SP2_OK;
}

int join_beside(sp2_handle_t h) {
  if (!h->side_pending) return SP2_OK;
  CK(cudaStreamWaitEvent(h->stream, h->side_ev[1], 0));
  h->side_pending = false;
  return SP2_OK;
}

size_t dsize(int dtype) { return dtype == SP2_F64 ? 8 : 4; }

// --------------------------------------------------------------- tile lists
void tile_shape(sp2_handle_t h, int mode, int64_t np, int* bm, int* bn) {
  if (split_mode(mode)) tc_tile_shape(h->tune.pair, bm, bn);
  else simt_tile_shape(mode, np, bm, bn);
}

// partials per output tile: a CTA pair's two CTAs each report their own rows
int parts_per_tile(sp2_handle_t h, int mode) { return split_mode(mode) && h->tune.pair ? 2 : 1; }

// Output tiles of a (rows x np) product in an L2-friendly order: groups of 8
// row blocks sweep the column blocks together, so CTAs resident at the same
// time share their operand slices. upper=true keeps only tiles that meet the
// upper triangle (row0 <= last column), which suffices for symmetric results.
int tile_list(sp2_handle_t h, int mode, int64_t rows, int64_t np, bool upper, const Tile** d,
              int* n) {
  int bm, bn;
  tile_shape(h, mode, np, &bm, &bn);
  char key[96];
  snprintf(key, sizeof key, "%d/%lld/%lld/%d/%dx%d", mode, (long long)rows, (long long)np,
           (int)upper, bm, bn);
  auto it = h->tiles.find(key);
  if (it != h->tiles.end()) {
    *d = it->second.d;
    *n = it->second.n;
    return SP2_OK;
  }
  std::vector<Tile> v;
  const int64_t nm = rows / bm, nn = np / bn;
  const int64_t G = 8;
  for (int64_t g0 = 0; g0 < nm; g0 += G) {
    const int64_t gs = (nm - g0) < G ? (nm - g0) : G;
    for (int64_t cn = 0; cn < nn; ++cn)
      for (int64_t m = g0; m < g0 + gs; ++m) {
        const int64_t r0 = m * bm, c0 = cn * bn;
        if (upper && r0 % np > c0 + bn - 1) continue;   // row within its batch entry
        v.push_back(Tile{(int)r0, (int)c0});
      }
  }
  Tile* dp = nullptr;
  CK(cudaMalloc(&dp, v.size() * sizeof(Tile) + 16));
  CK(cudaMemcpy(dp, v.data(), v.size() * sizeof(Tile), cudaMemcpyHostToDevice));
  h->tiles[key] = sp2_handle_s::TileList{dp, (int)v.size()};
  *d = dp;
  *n = (int)v.size();
  return SP2_OK;
}

// --------------------------------------------------------------- products
struct Ctx {
  sp2_handle_t h;
  int mode;
  int64_t n;      // caller's matrix size
  int64_t np;     // padded size
  DevState* st;
  Part3* part;    // trace / idempotency partials (>= max tiles)
  int64_t launches = 0;   // product launches that did work
  double flops = 0.0;     // executed product flops
  double alg = 0.0;       // algorithmic product flops
  int64_t kernels = 0;    // every kernel launched
  bool timing = false;
  int tail = 0;           // split-tail mode (product kernels read st->plane1)
  std::vector<std::pair<int, int>> timed;  // (step, event-pair index) per timed product launch
};

int ev_pair(Ctx& c, cudaEvent_t* a, cudaEvent_t* b) {
  sp2_handle_t h = c.h;
  const size_t i = c.timed.size();
  while (h->events.size() < 2 * (i + 1)) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    h->events.push_back(e);
  }
  *a = h->events[2 * i];
  *b = h->events[2 * i + 1];
  return SP2_OK;
}

// summed duration of the timed product launches of steps <= m
double timed_ms(Ctx& c, int m) {
  double tot = 0.0;
  for (size_t i = 0; i < c.timed.size(); ++i) {
    if (c.timed[i].first > m) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c.h->events[2 * i], c.h->events[2 * i + 1]) == cudaSuccess)
      tot += ms;
    else
      cudaGetLastError();
  }
  return tot;
}

int64_t timed_count(const Ctx& c, int m) {
  int64_t k = 0;
  for (auto& t : c.timed) k += t.first <= m ? 1 : 0;
  return k;
}

// tensor products per logical product: 3 (two planes), 6 (BF16X3), 1 (plain)
double k_mult(int mode) { return n_planes(mode) == 3 ? 6.0 : (split_mode(mode) ? 3.0 : 1.0); }

// settings shared by every product launch of a context: mode, padded size, state,
// partials and the handle's launch settings
int tc_common(Ctx& c, TcLaunch* L, int ntiles) {
  L->mode = c.mode;
  L->np = c.np;
  L->st = c.st;
  L->part = c.part;
  L->ntiles = ntiles;
  L->tune = c.h->tune;
  L->tail = c.tail;
  return SP2_OK;
}

// X_{n+1} = sigma_n>0 ? X_n^2 : 2 X_n - X_n^2, with trace partials; returns #partials.
// dec (CUDA-core modes): the step decision with these parameters is taken by the
// product's last block instead of a separate launch (dec->nparts is set here).
int square_step(Ctx& c, const MatBuf& xin, const MatBuf& xout, int step, int* nparts,
                const DecideParams* dec = nullptr) {
  sp2_handle_t h = c.h;
  const Tile* tl;
  int nt;
  TRY(tile_list(h, c.mode, c.np, c.np, true, &tl, &nt));
  int bm, bn;
  tile_shape(h, c.mode, c.np, &bm, &bn);
  TcLaunch L;   // workspace first: nothing is allocated inside the timed interval
  if (split_mode(c.mode)) TRY(tc_common(c, &L, nt));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c.timing) {
    TRY(ev_pair(c, &e0, &e1));
    CK(cudaEventRecord(e0, h->stream));
  }
  if (split_mode(c.mode)) {
    char eb[256] = {0};
    L.epi = EPI_SQUARE;
    L.P = TcOperand{xin.hi, xin.lo, c.np, xin.mid};
    L.Q = L.P;
    L.out = xout;
    L.prev = static_cast<const float*>(xin.master);
    L.tiles = tl;
    L.step = step;
    cudaError_t e = launch_gemm_tc(L, h->stream, eb, sizeof eb);
    if (e != cudaSuccess) return fail(h, SP2_ECUDA, "square product: %s %s", cudaGetErrorString(e), eb);
  } else {
    SimtDecide sd;
    if (dec) {
      void* dn;
      TRY(ws(h, "decide.done", sizeof(unsigned), &dn));
      sd.p = *dec;
      sd.p.nparts = nt;
      sd.st = c.st;
      sd.done = static_cast<unsigned*>(dn);
    }
    CK(launch_gemm_simt(c.mode, EPI_SQUARE, xin.master, c.np, xin.master, c.np, xout.master,
                        xin.master, c.part, tl, nt, c.st, step, h->stream, dec ? &sd : nullptr));
  }
  if (c.timing) {
    CK(cudaEventRecord(e1, h->stream));
    c.timed.push_back({step, 0});
  }
  c.launches++;
  c.kernels++;
  c.flops += 2.0 * bm * bn * (double)c.np * k_mult(c.mode) * nt;
  c.alg += (double)c.n * (double)(c.n + 1) * (double)c.n * k_mult(c.mode);
  *nparts = nt * parts_per_tile(h, c.mode);
  return SP2_OK;
}

// Workspace of the block-sparse recursion at padded size np.
int sparse_bufs(sp2_handle_t h, int64_t np, double tau, SparseBufs* B) {
  const int nb = (int)(np / 256);
  const size_t nt = (size_t)nb * (nb + 1) / 2;
  B->nb = nb;
  B->tau2 = tau * tau;
  void* p;
  for (int i = 0; i < 2; ++i) {
    const std::string k = std::to_string(i);
    TRY(ws(h, "sp.mask" + k, (size_t)nb * nb, &p));
    B->mask[i] = static_cast<uint8_t*>(p);
    TRY(ws(h, "sp.tiles" + k, nt * sizeof(Tile), &p));
    B->tiles[i] = static_cast<Tile*>(p);
    TRY(ws(h, "sp.ntiles" + k, sizeof(int), &p));
    B->ntiles[i] = static_cast<int*>(p);
    TRY(ws(h, "sp.kcnt" + k, nt * sizeof(int), &p));
    B->kcnt[i] = static_cast<int*>(p);
    TRY(ws(h, "sp.klist" + k, nt * nb * sizeof(uint16_t), &p));
    B->klist[i] = static_cast<uint16_t*>(p);
  }
  TRY(ws(h, "sp.zero", nt * sizeof(uint32_t), &p));
  B->zero = static_cast<uint32_t*>(p);
  TRY(ws(h, "sp.nzero", sizeof(int), &p));
  B->nzero = static_cast<int*>(p);
  TRY(ws(h, "sp.nrm2", (size_t)nb * nb * sizeof(double), &p));
  B->nrm2 = static_cast<double*>(p);
  TRY(ws(h, "sp.psum", sizeof(Part3), &p));
  B->psum = static_cast<Part3*>(p);
  return SP2_OK;
}

// The block-sparse square of `step` over the tiles and K lists the plan wrote
// into tiles[step % 2] (their count on the device); two partials per tile.
int sparse_square(Ctx& c, const MatBuf& xin, const MatBuf& xout, int step, const SparseBufs& B) {
  sp2_handle_t h = c.h;
  const int tl = step % 2;
  TcLaunch L;
  TRY(tc_common(c, &L, B.nb * (B.nb + 1) / 2));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c.timing) {
    TRY(ev_pair(c, &e0, &e1));
    CK(cudaEventRecord(e0, h->stream));
  }
  char eb[256] = {0};
  L.epi = EPI_SQUARE;
  L.P = TcOperand{xin.hi, xin.lo, c.np, xin.mid};
  L.Q = L.P;
  L.out = xout;
  L.prev = static_cast<const float*>(xin.master);
  L.tiles = B.tiles[tl];
  L.step = step;
  L.dyn_ntiles = B.ntiles[tl];
  L.kcnt = B.kcnt[tl];
  L.klist = B.klist[tl];
  L.nbk = B.nb;
  cudaError_t e = launch_gemm_tc(L, h->stream, eb, sizeof eb);
  if (e != cudaSuccess) return fail(h, SP2_ECUDA, "block-sparse square: %s %s", cudaGetErrorString(e), eb);
  if (c.timing) {
    CK(cudaEventRecord(e1, h->stream));
    c.timed.push_back({step, 0});
  }
  c.launches++;
  c.kernels++;
  return SP2_OK;
}

// Y_{n+1} = (1 - sigma_n) Y_n + sigma_n (Y_n X_n + X_n Y_n) for a batch of Y.
// Default: Z = Y X (tcgen05 EPI_PLAIN in split modes, CUDA cores otherwise), then
// the transpose-add kernel. With the handle's fused_response option (split modes):
// one tcgen05 launch over the upper tiles of every batch entry with the update in
// its epilogue (EPI_SYMM, no Z); in FP16X2 the output planes then take the scale
// sc.yscale[slot_out], fixed beforehand from ||Y_n||_F, and the scale of Y_{n+2}
// (slot_in) follows from this launch's partials.
int response_step(Ctx& c, const MatBuf& x, const MatBuf& yin, const MatBuf& yout, int64_t batch,
                  int step, const ScaleBuf& sc, int slot_in, int slot_out) {
  sp2_handle_t h = c.h;
  const int64_t rows = batch * c.np;
  const bool split = split_mode(c.mode);
  const bool fused = split && h->tune.fused_response;
  const Tile* tl;
  int nt;
  TRY(tile_list(h, c.mode, rows, c.np, fused, &tl, &nt));
  int bm, bn;
  tile_shape(h, c.mode, c.np, &bm, &bn);
  // workspace first: nothing is allocated inside the timed interval
  TcLaunch L;
  void* yp = nullptr;
  void* z = nullptr;
  if (fused) {
    TRY(ws(h, "ypart", (size_t)nt * parts_per_tile(h, c.mode) * sizeof(Part3), &yp));
  } else {
    TRY(ws(h, "Z", (size_t)rows * c.np * master_size(c.mode), &z));
  }
  if (split) TRY(tc_common(c, &L, nt));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c.timing) {
    TRY(ev_pair(c, &e0, &e1));
    CK(cudaEventRecord(e0, h->stream));
  }
  const bool f16 = c.mode == SP2_MODE_FP16X2;
  if (fused) {
    char eb[256] = {0};
    L.epi = EPI_SYMM;
    L.P = TcOperand{yin.hi, yin.lo, rows, yin.mid};
    L.Q = TcOperand{x.hi, x.lo, c.np, x.mid};
    L.out = yout;
    L.prev = static_cast<const float*>(yin.master);
    L.part = static_cast<Part3*>(yp);
    L.tiles = tl;
    L.step = step;
    if (f16) {
      L.p_scale = sc.yscale + slot_in * sc.B;
      L.o_scale = sc.yscale + slot_out * sc.B;
    }
    cudaError_t e = launch_gemm_tc(L, h->stream, eb, sizeof eb);
    if (e != cudaSuccess) return fail(h, SP2_ECUDA, "response product: %s %s", cudaGetErrorString(e), eb);
    if (c.timing) {
      CK(cudaEventRecord(e1, h->stream));
      c.timed.push_back({step, 0});
    }
    if (f16) {
      CK(launch_sym_scale(static_cast<Part3*>(yp), parts_per_tile(h, c.mode), tl, nt, c.np, batch,
                          c.st, step,
                          sc.yscale + slot_in * sc.B, h->stream));
      c.kernels++;
    }
    c.launches++;
    c.kernels++;
    // the update takes Y X + X Y over the upper tiles: K = 2 np per output tile
    c.flops += 2.0 * bm * bn * (double)c.np * 2.0 * k_mult(c.mode) * nt;
    c.alg += 2.0 * (double)batch * (double)c.n * (double)c.n * (double)c.n * k_mult(c.mode);
    return SP2_OK;
  }
  if (split) {
    char eb[256] = {0};
    if (f16) CK(cudaMemsetAsync(sc.zmax, 0, sizeof(float) * batch, h->stream));
    L.epi = EPI_PLAIN;
    L.P = TcOperand{yin.hi, yin.lo, rows, yin.mid};
    L.Q = TcOperand{x.hi, x.lo, c.np, x.mid};
    MatBuf zo;
    zo.master = z;
    L.out = zo;
    L.tiles = tl;
    L.step = step;
    if (f16) {
      L.p_scale = sc.yscale + slot_in * sc.B;
      L.zmax = sc.zmax;
    }
    cudaError_t e = launch_gemm_tc(L, h->stream, eb, sizeof eb);
    if (e != cudaSuccess) return fail(h, SP2_ECUDA, "response product: %s %s", cudaGetErrorString(e), eb);
  } else {
    CK(launch_gemm_simt(c.mode, EPI_PLAIN, yin.master, rows, x.master, c.np, z, nullptr, c.part,
                        tl, nt, c.st, step, h->stream));
  }
  if (c.timing) {
    CK(cudaEventRecord(e1, h->stream));
    c.timed.push_back({step, 0});
  }
  if (f16) CK(cudaMemsetAsync(sc.ymax + slot_out * sc.B, 0, sizeof(float) * batch, h->stream));
  CK(launch_symm_update(z, yin, yout, c.np, batch, c.mode, c.st, step, sc, slot_in, slot_out,
                        h->stream));
  c.launches++;
  c.kernels += 2;
  c.flops += 2.0 * bm * bn * (double)c.np * k_mult(c.mode) * nt;
  c.alg += 2.0 * (double)batch * (double)c.n * (double)c.n * (double)c.n * k_mult(c.mode);
  return SP2_OK;
}

// FP16X2: the plane scale of the first response step's output (slot `slot_out`)
// from the Frobenius norms of the batch in `m` (the response update at most
// doubles the 2-norm)
int first_sym_scale(Ctx& c, const MatBuf& m, int64_t batch, const ScaleBuf& sc, int slot_out) {
  sp2_handle_t h = c.h;
  const int np_ = fro_nparts();
  void* fp;
  TRY(ws(h, "fro.part", (size_t)batch * np_ * sizeof(double), &fp));
  CK(launch_fro_scale(static_cast<const float*>(m.master), c.np, batch, static_cast<double*>(fp),
                      np_, sc.yscale + slot_out * sc.B, h->stream));
  c.kernels += 2;
  return SP2_OK;
}

// With every X_n kept (k = 1) in a split mode, the checkpoint holds the hi/lo planes
// (np^2 x 4 bytes, the size of the FP32 master) instead of the master.
bool ckpt_planes(int mode, int k) { return k == 1 && n_planes(mode) == 2; }

// SP2_CKPT_AUTO: the smallest checkpoint interval k whose kept history fits in device
// memory next to the working set, so X_n is recomputed only when the history of
// max_iter steps would outgrow it. Working set reserved: X ping-pong, the adjoint's G
// ping-pong and product output for `batch` matrices, the k-step segment and 1 GiB.
int resolve_ckpt(sp2_handle_t h, sp2_opts* o, int64_t np, int64_t batch) {
  if (o->ckpt_k != SP2_CKPT_AUTO) return SP2_OK;
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  double avail = (double)fr;
  if (h->limit) avail = std::min(avail, (double)h->limit - (double)h->held);
  const double el = (double)np * (double)np;
  const double ms = (double)master_size(o->mode), mat_b = el * (ms + 2.0 * n_planes(o->mode));
  const double b = (double)(batch > 0 ? batch : 1);
  avail -= 2.0 * mat_b + 2.0 * b * mat_b + b * el * ms + (double)(1ull << 30);
  const int cap = o->fixed_m > 0 ? o->fixed_m : o->max_iter;
  int k = cap;
  for (int kk = 1; kk <= cap; ++kk) {
    const double need = (double)((cap + kk - 1) / kk) * el * ms + (double)(kk - 1) * mat_b;
    if (need <= avail) {
      k = kk;
      break;
    }
  }
  o->ckpt_k = k;
  return SP2_OK;
}

int validate_opts(sp2_handle_t h, const sp2_opts* o) {
  if (o->mode != SP2_MODE_FP64 && o->mode != SP2_MODE_FP32 && o->mode != SP2_MODE_BF16X2 &&
      o->mode != SP2_MODE_FP16X2 && o->mode != SP2_MODE_BF16X3)
    return fail(h, SP2_EINVAL, "unknown mode %d", o->mode);
  if (o->max_iter < 1 || o->max_iter > SP2_MAX_ITER)
    return fail(h, SP2_EINVAL, "max_iter %d outside 1..%d", o->max_iter, SP2_MAX_ITER);
  if (o->fixed_m > SP2_MAX_ITER) return fail(h, SP2_EINVAL, "fixed_m > %d", SP2_MAX_ITER);
  if (o->fixed_m > 0 && !o->sigma_in) return fail(h, SP2_EINVAL, "fixed_m without sigma_in");
  if (o->fixed_m > 0)
    for (int i = 0; i < o->fixed_m; ++i)
      if (o->sigma_in[i] != 1 && o->sigma_in[i] != -1)
        return fail(h, SP2_EINVAL, "sigma_in[%d] = %d is not +-1", i, (int)o->sigma_in[i]);
  if (o->ckpt_k < 1 && o->ckpt_k != SP2_CKPT_AUTO)
    return fail(h, SP2_EINVAL, "ckpt_k must be >= 1 or SP2_CKPT_AUTO");
  if (!(o->tail_f >= 0.0)) return fail(h, SP2_EINVAL, "tail_f must be >= 0");
  if (o->block_sparse && !(o->block_tau >= 0.0 && !std::isinf(o->block_tau)))
    return fail(h, SP2_EINVAL, "block_tau must be finite and >= 0");
  return SP2_OK;
}

sp2_opts resolve(const sp2_opts* in) {
  sp2_opts o;
  sp2_default_opts(&o);
  if (in) o = *in;
  if (o.max_iter == 0) o.max_iter = 100;
  if (o.min_iter < 0) o.min_iter = 4;
  if (o.floor_gate < 0) o.floor_gate = 0.03;
  if (o.ckpt_k == 0) o.ckpt_k = 4;
  // the named bfloat16-bulk / split-tail mode is BF16X2 with the split tail on
  if (o.mode == SP2_MODE_BF16_TAIL) {
    o.mode = SP2_MODE_BF16X2;
    if (o.tail_f == 0.0) o.tail_f = SP2_DEFAULT_TAIL_F;
  }
  return o;
}

int check_common(sp2_handle_t h, const void* H, int64_t N, int dtype, double nocc) {
  if (!h) return SP2_EINVAL;
  if (N < 0) return fail(h, SP2_EINVAL, "N = %lld < 0", (long long)N);
  if (N > (int64_t)1 << 20) return fail(h, SP2_EINVAL, "N = %lld too large", (long long)N);
  if (dtype != SP2_F64 && dtype != SP2_F32) return fail(h, SP2_EINVAL, "unknown dtype %d", dtype);
  if (N > 0 && !H) return fail(h, SP2_EINVAL, "H is NULL");
  if (!(nocc >= 0.0 && nocc <= (double)N)) return fail(h, SP2_EINVAL, "nocc %g outside [0, N]", nocc);
  return SP2_OK;
}

int poll_state(sp2_handle_t h) {
  CK(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->h_state->abort_flag)
    return fail(h, SP2_ETIMEOUT, "a device-side wait timed out in a product kernel");
  return SP2_OK;
}

// enqueue a snapshot of the state's trailing part into ring slot `step` % kRing
int ring_record(sp2_handle_t h, int step) {
  const int slot = step % sp2_handle_s::kRing;
  const size_t off = devstate_tail_offset();
  CK(cudaMemcpyAsync(reinterpret_cast<char*>(h->ring + slot) + off,
                     reinterpret_cast<const char*>(h->d_state) + off, sizeof(DevState) - off,
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaEventRecord(h->ring_ev[slot], h->stream));
  return SP2_OK;
}

// wait for the snapshot of `step` and return it
int ring_read(sp2_handle_t h, int step, const DevState** out) {
  const int slot = step % sp2_handle_s::kRing;
  CK(cudaEventSynchronize(h->ring_ev[slot]));
  *out = h->ring + slot;
  return SP2_OK;
}

// --------------------------------------------------------------- the SP2 driver
struct Sp2Out {
  int M = 0;
  bool converged = false;
  double alpha = 0, beta = 0, emin = 0, emax = 0;
  MatBuf xout;    // X_{M+1} (the kept floor candidate when the stop backtracked: master only)
  MatBuf yout;    // Y_{M+1}, likewise
  int stop_step = 0;  // the step after which the stop test fired (>= M)
  bool sparse = false;   // block-sparse recursion (info reports the formed block share)
};

// Runs Eq. DM0 on the padded X_1 = alpha I + beta H. If ybatch > 0, the
// response Y of Eq. DMPert / DMSuscept is carried along (merged form,
// Appendix), starting from Y_1 = beta B. If keep, X_n is checkpointed every
// ckpt_k steps for the adjoint.
// The spectral bounds, alpha and beta are computed on the device; the host
// enqueues step after step and learns of the stop from the snapshot ring, at
// most kLookahead steps behind, so it never waits for the GPU to drain. On return
// the stop (M, the kept iterate) is known; the GPU may still be running the last
// steps (no-ops past the stop).
int run_sp2(sp2_handle_t h, const void* Hd, int64_t n, int dtype, double nocc, const sp2_opts& o,
            const void* Bd, int64_t ybatch, int b_diag, bool keep, MatBuf X[2], MatBuf Y[2],
            Ctx& c, Sp2Out* out) {
  const int64_t np = c.np;   // the caller's padding (one for every mode a loop may switch to)
  const int mode = o.mode;
  const bool sparse = o.block_sparse != 0;
  if (sparse) {
    if (!split_mode(mode) || !h->tune.pair)
      return fail(h, SP2_EINVAL, "block_sparse: the squares run in the split modes on CTA pairs");
    if (ybatch > 0 || keep)
      return fail(h, SP2_EINVAL, "block_sparse: sp2_density without keep_history only");
    if (o.tail_f > 0.0) return fail(h, SP2_EINVAL, "block_sparse with tail_f > 0");
    if (np / 256 > kMaxSparseBlocks)
      return fail(h, SP2_EINVAL, "block_sparse: N above %d", 256 * kMaxSparseBlocks);
  }
  CK(cudaMemsetAsync(h->d_state, 0, sizeof(DevState), h->stream));
  // spectral bounds (Sec. II) and X_1 = alpha I + beta H, on the device
  if (o.eps_min < o.eps_max) {
    CK(launch_set_bounds(h->d_state, o.eps_min, o.eps_max, h->stream));
    c.kernels++;
  } else {
    const int nb = bounds_nparts(n);
    void* bp;
    TRY(ws(h, "bounds.part", nb * sizeof(double2), &bp));
    CK(launch_bounds(Hd, n, dtype, static_cast<double2*>(bp), nb, h->d_state, h->stream));
    c.kernels += 2;
  }
  if (o.fixed_m > 0) {
    CK(launch_set_sigma(h->d_state, o.sigma_in, o.fixed_m, h->stream));
    c.kernels++;
  }

  TRY(mat(h, "X0", np, np, mode, &X[0]));
  TRY(mat(h, "X1", np, np, mode, &X[1]));
  const int ni = init_nparts(np);
  CK(launch_init(Hd, n, np, 1, dtype, 0, 0, 0.0, 0.0, mode, X[1], c.part, ni, nullptr, h->stream,
                 INIT_STATE, h->d_state));
  c.kernels++;
  DecideParams dp;
  dp.nocc = nocc;
  dp.idem_tol = o.idem_tol;
  dp.floor_gate = o.floor_gate;
  dp.min_iter = o.min_iter;
  dp.max_iter = o.max_iter;
  dp.fixed_m = o.fixed_m;
  dp.tail_f = split_mode(mode) ? o.tail_f : 0.0;
  c.tail = dp.tail_f > 0.0 ? 1 : 0;
  dp.n = 1;
  dp.nparts = ni;
  SparseBufs sb;
  if (sparse) {
    // X~_1 = T_tau(X_1); the first square's tiles; X[0]'s content is unknown, so
    // every block of it counts as stale for the first square
    TRY(sparse_bufs(h, np, o.block_tau, &sb));
    CK(launch_block_norms(static_cast<const float*>(X[1].master), np, sb.nb, sb.nrm2, h->stream));
    CK(cudaMemsetAsync(sb.mask[0], 1, (size_t)sb.nb * sb.nb, h->stream));
    CK(launch_sparse_plan(sb, 1, 1, 0, 1, c.part, ni, c.st, 0, h->stream));
    CK(launch_zero_blocks(sb, X[1], np, mode, c.st, 0, 1, h->stream));
    c.kernels += 3;
    dp.nparts = 1;
    dp.ratio_floor = 1;
    CK(launch_decide(sb.psum, c.st, dp, h->stream));
  } else {
    CK(launch_decide(c.part, c.st, dp, h->stream));
  }
  c.kernels++;
  ScaleBuf sc;
  if (ybatch > 0) {
    TRY(mat(h, "Y0", ybatch * np, np, mode, &Y[0]));
    TRY(mat(h, "Y1", ybatch * np, np, mode, &Y[1]));
    const bool f16 = mode == SP2_MODE_FP16X2;
    if (f16) {
      TRY(scales(h, "Y.scale", ybatch, &sc));
      CK(cudaMemsetAsync(sc.ymax, 0, sizeof(float) * 2 * ybatch, h->stream));
    }
    CK(launch_init(Bd, n, np, ybatch, dtype, b_diag, 0, 0.0, 0.0, mode, Y[1], nullptr, 0,
                   f16 ? sc.ymax + 1 * ybatch : nullptr, h->stream, INIT_STATE_BETA, h->d_state));
    c.kernels++;
    if (f16) {
      CK(launch_split_scaled(Y[1], np, sc, 1, h->stream));
      c.kernels += 2;
      if (h->tune.fused_response) TRY(first_sym_scale(c, Y[1], ybatch, sc, 0));
    }
  }

  const int maxit = o.fixed_m > 0 ? o.fixed_m : o.max_iter;
  const size_t xbytes = (size_t)np * np * master_size(mode);
  const double f0 = c.flops, a0 = c.alg;
  const int64_t l0 = c.launches;
  double fstep = 0.0, astep = 0.0;
  int64_t lstep = 0;
  // the floor candidate with the smallest f so far (the result when the floor test fires)
  const bool track = o.floor_gate > 0.0 && o.fixed_m == 0;
  MatBuf xbest, ybest;
  if (track) {
    TRY(ws(h, "Xbest.m", xbytes, &xbest.master));
    if (ybatch > 0) TRY(ws(h, "Ybest.m", (size_t)ybatch * xbytes, &ybest.master));
  }
  if (!split_mode(mode) && !sparse) {
    // the completion counter of the squares' last-block decision starts at zero
    void* dn;
    TRY(ws(h, "decide.done", sizeof(unsigned), &dn));
    CK(cudaMemsetAsync(dn, 0, sizeof(unsigned), h->stream));
  }
  const DevState* seen = nullptr;   // latest snapshot read
  int last = 0;                     // last step enqueued
  for (int step = 1; step <= maxit; ++step) {
    const MatBuf& xin = X[step % 2];
    const MatBuf& xo = X[(step + 1) % 2];
    if (keep && (step - 1) % o.ckpt_k == 0) {
      void* ck;
      TRY(ws(h, "ckpt." + std::to_string((step - 1) / o.ckpt_k), xbytes, &ck));
      if (ckpt_planes(mode, o.ckpt_k)) {
        // every X_n kept: its 16-bit planes are all the adjoint products read
        const size_t pb = (size_t)np * np * 2;
        CK(cudaMemcpyAsync(ck, xin.hi, pb, cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(static_cast<char*>(ck) + pb, xin.lo, pb, cudaMemcpyDeviceToDevice,
                           h->stream));
      } else {
        CK(cudaMemcpyAsync(ck, xin.master, xbytes, cudaMemcpyDeviceToDevice, h->stream));
      }
    }
    if (ybatch > 0)
      TRY(response_step(c, xin, Y[step % 2], Y[(step + 1) % 2], ybatch, step, sc, step % 2,
                        (step + 1) % 2));
    dp.n = step + 1;
    if (sparse) {
      TRY(sparse_square(c, xin, xo, step, sb));
      CK(launch_sparse_plan(sb, 0, (step + 1) % 2, step % 2, (step + 1) % 2, c.part, 0, c.st, step,
                            h->stream));
      CK(launch_zero_blocks(sb, xo, np, mode, c.st, step, 0, h->stream));
      c.kernels += 2;
      CK(launch_decide(sb.psum, c.st, dp, h->stream));
      c.kernels++;
    } else if (!split_mode(mode)) {
      // CUDA-core square: its last block takes the decision
      int nparts = 0;
      TRY(square_step(c, xin, xo, step, &nparts, &dp));
      dp.nparts = nparts;
    } else {
      int nparts = 0;
      TRY(square_step(c, xin, xo, step, &nparts));
      dp.nparts = nparts;
      CK(launch_decide(c.part, c.st, dp, h->stream));
      c.kernels++;
    }
    if (track) {
      CK(launch_keep_best(xin.master, xbest.master, np * np, mode, c.st, step, h->stream));
      c.kernels++;
      if (ybatch > 0) {
        CK(launch_keep_best(Y[step % 2].master, ybest.master, ybatch * np * np, mode, c.st, step,
                            h->stream));
        c.kernels++;
      }
    }
    if (step == 1) {
      fstep = c.flops - f0;
      astep = c.alg - a0;
      lstep = c.launches - l0;
    }
    TRY(ring_record(h, step));
    last = step;
    if (step > sp2_handle_s::kLookahead) {
      TRY(ring_read(h, step - sp2_handle_s::kLookahead, &seen));
      if (seen->stop_at != 0 || seen->abort_flag) break;
    }
  }
  if (!seen || (seen->stop_at == 0 && !seen->abort_flag)) TRY(ring_read(h, last, &seen));
  const DevState& S = *seen;
  out->alpha = S.alpha;
  out->beta = S.beta;
  out->emin = S.bounds[0];
  out->emax = S.bounds[1];
  if (S.abort_flag) return fail(h, SP2_ETIMEOUT, "a device-side wait timed out in a product kernel");
  if (S.nonfinite) {
    if (S.stop_at < 0) return fail(h, SP2_ENONFINITE, "non-finite spectral bounds (NaN/Inf in H)");
    return fail(h, SP2_ENONFINITE, "non-finite trace after step %d", S.stop_at);
  }
  const bool stopped = S.stop_at > 0;
  const int M = stopped ? S.stop_at : maxit;
  out->M = M;
  out->converged = stopped;
  const bool back = stopped && S.backtracked;
  out->xout = back ? xbest : X[(M + 1) % 2];
  out->yout = back ? ybest : Y[(M + 1) % 2];
  out->stop_step = stopped ? S.stop_step : M;
  if (out->stop_step < M) out->stop_step = M;
  // executed-work accounting covers only the steps that ran (later launches were no-ops)
  c.flops = f0 + fstep * out->stop_step;
  c.alg = a0 + astep * out->stop_step;
  c.launches = l0 + lstep * out->stop_step;
  if (sparse) {
    // per listed K block of a 256 x 256 tile: 256^3 products of every split term
    const double w = S.work_kblocks * 2.0 * 256.0 * 256.0 * 256.0 * k_mult(mode);
    c.flops = f0 + w;
    c.alg = a0 + w;
    out->sparse = true;
  }
  return SP2_OK;
}

void fill_info(sp2_handle_t h, const Sp2Out& r, const Ctx& c, sp2_info* info) {
  if (!info) return;
  memset(info, 0, sizeof *info);
  info->M = r.M;
  info->converged = r.converged ? 1 : 0;
  info->alpha = r.alpha;
  info->beta = r.beta;
  info->eps_min = r.emin;
  info->eps_max = r.emax;
  const DevState& s = *h->h_state;
  for (int i = 1; i <= r.M; ++i) info->sigma[i - 1] = (int8_t)s.sigma[i];
  for (int i = 1; i <= r.M + 1; ++i) info->errors[i - 1] = s.t1[i] - s.t2[i];
  for (int i = 1; i <= r.M; ++i) info->idem_fro[i - 1] = s.f[i];
  info->trace = s.t1[r.M + 1];
  info->idem_err = s.t1[r.M + 1] - s.t2[r.M + 1];
  for (int i = 1; i <= r.M; ++i) info->tail_single_steps += s.plane1[i] ? 1 : 0;
  if (r.sparse && r.M > 0) {
    // mean over the steps of the result (1..M) of the upper blocks each square formed
    double fs = 0.0;
    for (int i = 1; i <= r.M; ++i) fs += s.fill[i];
    info->block_fill = fs / r.M;
  }
  info->n_gemm_launches = c.launches;
  info->executed_flops = c.flops;
  info->algorithmic_flops = c.alg;
  info->kernel_launches = c.kernels;
}

// timing fields; call after the stream has been synchronised
void fill_timing(Ctx& c, int m, sp2_info* info) {
  if (!info) return;
  info->n_gemm_launches = c.launches;
  info->executed_flops = c.flops;
  info->algorithmic_flops = c.alg;
  info->kernel_launches = c.kernels;
  if (c.timing) {
    info->product_ms = timed_ms(c, m);
    info->product_launches_timed = timed_count(c, m);
  }
}

int make_ctx(sp2_handle_t h, int mode, int64_t n, int64_t np, bool timing, Ctx* c) {
  c->h = h;
  c->mode = mode;
  c->n = n;
  c->np = np;
  c->timing = timing;
  c->st = h->d_state;
  int bm, bn;
  tile_shape(h, mode, np, &bm, &bn);
  int64_t maxp = (np / bm) * (np / bn) * parts_per_tile(h, mode) + 8;
  if (maxp < init_nparts(np)) maxp = init_nparts(np);
  void* p;
  TRY(ws(h, "part", (size_t)maxp * sizeof(Part3), &p));
  c->part = static_cast<Part3*>(p);
  return SP2_OK;
}

// Eq. DM2 over the kept history: G_{M+1} = B, G_n = (1 - s_n) G_{n+1} + s_n (G_{n+1} X_n + X_n G_{n+1}),
// n = M..1; result beta * G_1. X_n is restored from the checkpoint of its
// segment and the segment is recomputed forward with the stored branches.
int run_adjoint(sp2_handle_t h, const void* Bd, int64_t batch, int b_diag, int symmetrize,
                int dtype, void* outd, int out_dtype, Ctx& c, DevState** adj_state) {
  auto& hs = h->hist;
  const int64_t np = hs.np, n = hs.n;
  const int mode = hs.mode, M = hs.M, k = hs.k;
  // the adjoint's own state: the branch signs of the kept forward recursion (a
  // device copy), with nothing to stop and no floor candidate to keep
  void* stp;
  void* hst;
  TRY(ws(h, "adj.state", sizeof(DevState), &stp));
  TRY(ws(h, "hist.state", sizeof(DevState), &hst));
  DevState* ast = static_cast<DevState*>(stp);
  CK(cudaMemcpyAsync(ast, hst, sizeof(DevState), cudaMemcpyDeviceToDevice, h->stream));
  CK(launch_adjoint_state(ast, h->stream));
  c.kernels++;
  c.st = ast;
  c.tail = hs.tail;   // the adjoint step n uses the planes its forward step n used
  *adj_state = ast;

  MatBuf G[2];
  TRY(mat(h, "G0", batch * np, np, mode, &G[0]));
  TRY(mat(h, "G1", batch * np, np, mode, &G[1]));
  int gs = (M + 1) % 2;  // slot of G_{M+1}
  ScaleBuf sc;
  const bool f16 = mode == SP2_MODE_FP16X2;
  if (f16) {
    TRY(scales(h, "G.scale", batch, &sc));
    CK(cudaMemsetAsync(sc.ymax, 0, sizeof(float) * 2 * batch, h->stream));
  }
  CK(launch_init(Bd, n, np, batch, dtype, b_diag, symmetrize, 0.0, 1.0, mode, G[gs], nullptr, 0,
                 f16 ? sc.ymax + gs * batch : nullptr, h->stream));
  c.kernels++;
  if (f16) {
    CK(launch_split_scaled(G[gs], np, sc, gs, h->stream));
    c.kernels += 2;
    if (h->tune.fused_response) TRY(first_sym_scale(c, G[gs], batch, sc, 1 - gs));
  }
  // segment buffers X_{s0+1} .. X_{s0+k-1}; X_{s0} is read from its checkpoint in place
  // (the master) with its planes split into seg[0], or taken as the kept planes
  const bool planes = ckpt_planes(mode, k);
  std::vector<MatBuf> seg(k);
  for (int i = 1; i < k; ++i) TRY(mat(h, "seg." + std::to_string(i), np, np, mode, &seg[i]));
  if (!planes && split_mode(mode)) {
    void* p;
    TRY(ws(h, "seg.0.h", (size_t)np * np * 2, &p));
    seg[0].hi = static_cast<uint16_t*>(p);
    TRY(ws(h, "seg.0.l", (size_t)np * np * 2, &p));
    seg[0].lo = static_cast<uint16_t*>(p);
    if (n_planes(mode) == 3) {
      TRY(ws(h, "seg.0.d", (size_t)np * np * 2, &p));
      seg[0].mid = static_cast<uint16_t*>(p);
    }
  }
  const size_t xbytes = (size_t)np * np * master_size(mode);
  const int nseg = (M + k - 1) / k;
  for (int j = nseg - 1; j >= 0; --j) {
    const int s0 = j * k + 1;
    const int s1 = (j * k + k) < M ? (j * k + k) : M;
    void* ck;
    TRY(ws(h, "ckpt." + std::to_string(j), xbytes, &ck));
    if (planes) {
      seg[0].master = nullptr;
      seg[0].hi = static_cast<uint16_t*>(ck);
      seg[0].lo = seg[0].hi + (size_t)np * np;
    } else {
      seg[0].master = ck;
      if (split_mode(mode)) {
        CK(launch_split(seg[0], np, np, mode, h->stream));
        c.kernels++;
      }
    }
    for (int s = s0; s < s1; ++s) {
      int nparts;
      TRY(square_step(c, seg[s - s0], seg[s - s0 + 1], s, &nparts));
    }
    for (int s = s1; s >= s0; --s) {
      TRY(response_step(c, seg[s - s0], G[gs], G[1 - gs], batch, s, sc, gs, 1 - gs));
      gs = 1 - gs;
    }
  }
  // gs now holds G_1
  CK(launch_copy_out(G[gs], n, np, batch, mode, hs.beta, outd, out_dtype, h->stream));
  c.kernels++;
  c.st = h->d_state;
  // a timed-out device wait of the adjoint's launches shows in its own state,
  // which the completion of the call reads
  return SP2_OK;
}

// keep the forward recursion's device state (branch signs) for a later adjoint
int keep_history(sp2_handle_t h, const Sp2Out& r, int64_t n, int64_t np, int mode, int k,
                 int tail) {
  void* hst;
  TRY(ws(h, "hist.state", sizeof(DevState), &hst));
  CK(cudaMemcpyAsync(hst, h->d_state, sizeof(DevState), cudaMemcpyDeviceToDevice, h->stream));
  auto& hs = h->hist;
  hs.valid = true;
  hs.n = n;
  hs.np = np;
  hs.mode = mode;
  hs.M = r.M;
  hs.k = k;
  hs.beta = r.beta;
  hs.tail = tail;
  hs.sigma.clear();   // filled when the call completes
  return SP2_OK;
}


// --------------------------------------------------------------- call completion
}  // namespace

// What a call left for its completion: the device state to read, the status
// known when it returned, and what its info reports.
struct sp2_handle_s::Pending {
  bool sp2 = false;               // a forward recursion ran: info from the device state
  bool adjoint = false;           // sp2_adjoint: info from the kept history
  Sp2Out r;
  Ctx c;
  int ckpt_k = 0;
  bool hist_sigma = false;        // fill the kept history's branch signs
  DevState* adj_state = nullptr;  // an adjoint ran: its abort flag
  int status = SP2_OK;            // known when the call returned (ENOCONV)
  std::string msg;
};

namespace {

void drop_pending(sp2_handle_t h) {
  delete h->pending;
  h->pending = nullptr;
}

// Waits for the handle's stream, reads the device state and completes the last
// call: its status (a timed-out wait of the adjoint shows only now) and its info.
int complete_pending(sp2_handle_t h, sp2_info* info) {
  sp2_handle_s::Pending* p = h->pending;
  h->pending = nullptr;
  CK(cudaStreamSynchronize(h->stream));
  if (!p) {
    if (info) memset(info, 0, sizeof *info);
    return SP2_OK;
  }
  int code = p->status;
  std::string msg = p->msg;
  cudaError_t e = cudaMemcpy(h->h_state, h->d_state, sizeof(DevState), cudaMemcpyDeviceToHost);
  int adj_abort = 0;
  if (e == cudaSuccess && p->adj_state)
    e = cudaMemcpy(&adj_abort, &p->adj_state->abort_flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    delete p;
    return fail(h, SP2_ECUDA, "reading the device state failed: %s", cudaGetErrorString(e));
  }
  if (adj_abort || (p->sp2 && h->h_state->abort_flag)) {
    code = SP2_ETIMEOUT;
    msg = "a device-side wait timed out in a product kernel";
  }
  auto& hs = h->hist;
  if (p->hist_sigma && hs.valid) {
    hs.sigma.assign(hs.M + 1, 0);
    for (int i = 1; i <= hs.M; ++i) hs.sigma[i] = h->h_state->sigma[i];
  }
  if (info) {
    if (p->sp2) {
      fill_info(h, p->r, p->c, info);
    } else {
      memset(info, 0, sizeof *info);
      if (p->adjoint) {
        info->M = hs.M;
        info->converged = 1;
        info->beta = hs.beta;
        void* hst;
        if (ws(h, "hist.state", sizeof(DevState), &hst) == SP2_OK &&
            cudaMemcpy(h->h_state, hst, sizeof(DevState), cudaMemcpyDeviceToHost) == cudaSuccess)
          for (int i = 1; i <= hs.M; ++i) info->sigma[i - 1] = (int8_t)h->h_state->sigma[i];
      }
    }
    fill_timing(p->c, p->adjoint ? hs.M : p->r.M, info);
    info->ckpt_k = p->ckpt_k;
  }
  delete p;
  if (code != SP2_OK) return fail(h, code, "%s", msg.c_str());
  return SP2_OK;
}

// Ends a call whose work is enqueued: it completes now when the caller wants info
// or gets results in host memory, else it returns at once and sp2_synchronize
// completes it.
int finish_call(sp2_handle_t h, sp2_handle_s::Pending* p, sp2_info* info, bool wait) {
  drop_pending(h);
  h->pending = p;
  if (wait || info) return complete_pending(h, info);
  if (p->status != SP2_OK) return fail(h, p->status, "%s", p->msg.c_str());
  return SP2_OK;
}

// --------------------------------------------------------------- finite temperature
// A padded matrix of the finite-temperature recursion with its plane scale
// (FP16X2: a power of two from its max; 1 otherwise) and max accumulator.
struct FMat {
  MatBuf m;
  float* scale = nullptr;  // device float (FP16X2)
  float* amax = nullptr;   // device float (FP16X2)
};

int fmat(sp2_handle_t h, const std::string& name, int64_t np, int mode, FMat* f) {
  TRY(mat(h, name, np, np, mode, &f->m));
  if (mode == SP2_MODE_FP16X2) {
    void* p;
    TRY(ws(h, name + ".s", 2 * sizeof(float), &p));
    f->scale = static_cast<float*>(p);
    f->amax = f->scale + 1;
  }
  return SP2_OK;
}

// hi/lo planes of f from its master (FP16X2: scale from f->amax)
int fplanes(Ctx& c, FMat& f) {
  sp2_handle_t h = c.h;
  if (c.mode == SP2_MODE_BF16X2 || c.mode == SP2_MODE_BF16X3) {
    CK(launch_split(f.m, c.np, c.np, c.mode, h->stream));
    c.kernels++;
  } else if (c.mode == SP2_MODE_FP16X2) {
    ScaleBuf sc;
    sc.ymax = f.amax;
    sc.yscale = f.scale;
    sc.B = 1;
    CK(launch_split_scaled(f.m, c.np, sc, 0, h->stream));
    c.kernels += 2;
  }
  return SP2_OK;
}

// C = L R for symmetric R (R's rows are the K-major operand); master only,
// plus C's max in FP16X2 (planes follow from fplanes when C is an operand)
int fprod(Ctx& c, FMat& C, const FMat& L, const FMat& R) {
  sp2_handle_t h = c.h;
  const Tile* tl;
  int nt;
  TRY(tile_list(h, c.mode, c.np, c.np, false, &tl, &nt));
  int bm, bn;
  tile_shape(h, c.mode, c.np, &bm, &bn);
  TcLaunch T;   // workspace first: nothing is allocated inside the timed interval
  if (split_mode(c.mode)) TRY(tc_common(c, &T, nt));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c.timing) {
    TRY(ev_pair(c, &e0, &e1));
    CK(cudaEventRecord(e0, h->stream));
  }
  if (split_mode(c.mode)) {
    const bool f16 = c.mode == SP2_MODE_FP16X2;
    if (f16) CK(cudaMemsetAsync(C.amax, 0, sizeof(float), h->stream));
    char eb[256] = {0};
    T.epi = EPI_PLAIN;
    T.P = TcOperand{L.m.hi, L.m.lo, c.np, L.m.mid};
    T.Q = TcOperand{R.m.hi, R.m.lo, c.np, R.m.mid};
    T.out = C.m;
    T.tiles = tl;
    T.step = 0;
    if (f16) {
      T.p_scale = L.scale;
      T.q_scale = R.scale;
      T.zmax = C.amax;
    }
    cudaError_t e = launch_gemm_tc(T, h->stream, eb, sizeof eb);
    if (e != cudaSuccess) return fail(h, SP2_ECUDA, "finite-T product: %s %s", cudaGetErrorString(e), eb);
  } else {
    CK(launch_gemm_simt(c.mode, EPI_PLAIN, L.m.master, c.np, R.m.master, c.np, C.m.master, nullptr,
                        c.part, tl, nt, c.st, 0, h->stream));
  }
  if (c.timing) {
    CK(cudaEventRecord(e1, h->stream));
    c.timed.push_back({0, 0});
  }
  c.launches++;
  c.kernels++;
  c.flops += 2.0 * bm * bn * (double)c.np * k_mult(c.mode) * nt;
  c.alg += 2.0 * (double)c.n * (double)c.n * (double)c.n * k_mult(c.mode);
  return SP2_OK;
}

// out = z1 (Z1 + Z1^T) + z2 (Z2 + Z2^T) + a A + id I, then planes when `planes`
int fcomb(Ctx& c, FMat& out, const FMat* Z1, double z1, const FMat* Z2, double z2,
          const FMat* A, double a, double id, bool planes) {
  sp2_handle_t h = c.h;
  const bool f16 = c.mode == SP2_MODE_FP16X2;
  if (f16) CK(cudaMemsetAsync(out.amax, 0, sizeof(float), h->stream));
  CK(launch_combine(c.mode, out.m.master, c.np, c.n, Z1 ? Z1->m.master : nullptr, z1,
                    Z2 ? Z2->m.master : nullptr, z2, A ? A->m.master : nullptr, a, id,
                    f16 ? out.amax : nullptr, h->stream));
  c.kernels++;
  if (planes) TRY(fplanes(c, out));
  return SP2_OK;
}

// Newton-Schulz iterations for Z = S^{-1} with spec(S) in [1, 1 + 4 b^2]:
// Z_0 = 2 / (2 + 4 b^2) I, error ratio r = 4 b^2 / (2 + 4 b^2) squared each
// iteration; enough iterations for r^(2^k) <= tol.
int ns_iterations(double b, double tol) {
  const double r = 4.0 * b * b / (2.0 + 4.0 * b * b);
  int k = 0;
  double e = r;
  while (e > tol && k < 12) {
    e = e * e;
    ++k;
  }
  return k;
}
}  // namespace

// ====================================================================== C ABI
extern "C" {

void sp2_default_opts(sp2_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->mode = SP2_MODE_FP32;
  o->idem_tol = 0.0;
  o->floor_gate = 0.03;
  o->max_iter = 100;
  o->min_iter = 4;
  o->fixed_m = 0;
  o->sigma_in = nullptr;
  o->eps_min = 0.0;
  o->eps_max = 0.0;
  o->ckpt_k = 4;
  o->keep_history = 0;
}

int sp2_create(sp2_handle_t* out, void* stream, size_t limit) {
  if (!out) return SP2_EINVAL;
  *out = nullptr;
  sp2_handle_t h = new sp2_handle_s();
  h->stream = static_cast<cudaStream_t>(stream);
  h->limit = limit;
  int code = SP2_OK;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaMalloc(&h->d_state, sizeof(DevState)) != cudaSuccess ||
      cudaMallocHost(&h->h_state, sizeof(DevState)) != cudaSuccess) {
    cudaGetLastError();
    code = SP2_ECUDA;
  }
  if (code == SP2_OK &&
      cudaMallocHost(&h->ring, sizeof(DevState) * sp2_handle_s::kRing) != cudaSuccess) {
    cudaGetLastError();
    code = SP2_ECUDA;
  }
  for (int i = 0; code == SP2_OK && i < sp2_handle_s::kRing; ++i)
    if (cudaEventCreateWithFlags(&h->ring_ev[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      code = SP2_ECUDA;
    }
  if (code != SP2_OK) {
    for (int i = 0; i < sp2_handle_s::kRing; ++i)
      if (h->ring_ev[i]) cudaEventDestroy(h->ring_ev[i]);
    if (h->ring) cudaFreeHost(h->ring);
    if (h->h_state) cudaFreeHost(h->h_state);
    if (h->d_state) cudaFree(h->d_state);
    delete h;
    return code;
  }
  memset(h->h_state, 0, sizeof(DevState));
  memset(h->ring, 0, sizeof(DevState) * sp2_handle_s::kRing);
  *out = h;
  return SP2_OK;
}

int sp2_destroy(sp2_handle_t h) {
  if (!h) return SP2_EINVAL;
  cudaStreamSynchronize(h->stream);
  for (auto& kv : h->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  for (auto& kv : h->tiles) cudaFree(kv.second.d);
  if (h->d_state) cudaFree(h->d_state);
  if (h->h_state) cudaFreeHost(h->h_state);
  for (int i = 0; i < sp2_handle_s::kRing; ++i)
    if (h->ring_ev[i]) cudaEventDestroy(h->ring_ev[i]);
  if (h->ring) cudaFreeHost(h->ring);
  if (h->side) {
    cudaStreamSynchronize(h->side);
    cudaStreamDestroy(h->side);
    cudaEventDestroy(h->side_ev[0]);
    cudaEventDestroy(h->side_ev[1]);
  }
  for (auto e : h->events) cudaEventDestroy(e);
  delete h->pending;
  delete h;
  return SP2_OK;
}

int sp2_synchronize(sp2_handle_t h, sp2_info* info) {
  if (!h) return SP2_EINVAL;
  return complete_pending(h, info);
}

int sp2_set_stream(sp2_handle_t h, void* stream) {
  if (!h) return SP2_EINVAL;
  h->stream = static_cast<cudaStream_t>(stream);
  return SP2_OK;
}

int sp2_set_option(sp2_handle_t h, int option, int64_t value) {
  if (!h) return SP2_EINVAL;
  switch (option) {
    case SP2_OPTION_WAIT_LIMIT_NS:
      if (value < 1000 || value > (int64_t)60000000000ll)
        return fail(h, SP2_EINVAL, "wait limit %lld ns outside [1e3, 6e10]", (long long)value);
      h->tune.wait_ns = (unsigned long long)value;
      return SP2_OK;
    case SP2_OPTION_WITHHOLD_LOAD:
      h->tune.withhold = value != 0 ? 1 : 0;
      return SP2_OK;
    case SP2_OPTION_FUSED_RESPONSE:
      h->tune.fused_response = value != 0 ? 1 : 0;
      return SP2_OK;
    case SP2_OPTION_PAIR_TILES:
      h->tune.pair = value != 0 ? 1 : 0;
      return SP2_OK;
    default:
      return fail(h, SP2_EINVAL, "unknown option %d", option);
  }
}

const char* sp2_last_error(sp2_handle_t h) { return h ? h->err.c_str() : "null handle"; }

size_t sp2_workspace_bytes(sp2_handle_t h) { return h ? h->held : 0; }

int sp2_density(sp2_handle_t h, const void* H, int64_t N, int dtype, double nocc,
                const sp2_opts* opts_in, void* D, sp2_info* info) {
  TRY(check_common(h, H, N, dtype, nocc));
  if (N > 0 && !D) return fail(h, SP2_EINVAL, "D is NULL");
  sp2_opts o = resolve(opts_in);
  TRY(validate_opts(h, &o));
  if (info) memset(info, 0, sizeof *info);
  if (N == 0) {
    if (info) info->converged = 1;
    return SP2_OK;
  }
  const size_t mb = (size_t)N * N * dsize(dtype);
  const void* Hd;
  TRY(stage_in(h, "H", H, mb, &Hd));
  OutStage od;
  TRY(stage_out(h, "D", D, mb, &od));
  const int64_t np = pad_n(N, o.mode);
  Ctx c;
  TRY(make_ctx(h, o.mode, N, np, o.time_kernels != 0, &c));
  MatBuf X[2], Y[2];
  Sp2Out r;
  const bool keep = o.keep_history != 0;
  if (keep) {
    h->hist.valid = false;
    TRY(resolve_ckpt(h, &o, np, 1));
  }
  TRY(run_sp2(h, Hd, N, dtype, nocc, o, nullptr, 0, 0, keep, X, Y, c, &r));
  CK(launch_copy_out(r.xout, N, np, 1, o.mode, 1.0, od.dev, dtype, h->stream));
  c.kernels++;
  TRY(finish_out(h, od));
  if (keep) TRY(keep_history(h, r, N, np, o.mode, o.ckpt_k, c.tail));
  auto* p = new sp2_handle_s::Pending();
  p->sp2 = true;
  p->r = r;
  p->c = c;
  p->ckpt_k = keep ? o.ckpt_k : 0;
  p->hist_sigma = keep;
  if (!r.converged) {
    p->status = SP2_ENOCONV;
    p->msg = "no convergence in " + std::to_string(r.M) + " steps";
  }
  return finish_call(h, p, info, od.host);
}

int sp2_response(sp2_handle_t h, const void* H, int64_t N, int dtype, double nocc, const void* H1,
                 int64_t K, int h1_diag_only, const sp2_opts* opts_in, void* D, void* D1,
                 sp2_info* info) {
  TRY(check_common(h, H, N, dtype, nocc));
  if (K < 0) return fail(h, SP2_EINVAL, "K < 0");
  if (N > 0 && K > 0 && (!H1 || !D1)) return fail(h, SP2_EINVAL, "H1 or D1 is NULL");
  sp2_opts o = resolve(opts_in);
  TRY(validate_opts(h, &o));
  if (info) memset(info, 0, sizeof *info);
  if (N == 0) {
    if (info) info->converged = 1;
    return SP2_OK;
  }
  const size_t mb = (size_t)N * N * dsize(dtype);
  const size_t b_bytes = (size_t)K * (h1_diag_only ? N : N * N) * dsize(dtype);
  const void *Hd, *Bd = nullptr;
  TRY(stage_in(h, "H", H, mb, &Hd));
  if (K > 0) TRY(stage_in(h, "B", H1, b_bytes, &Bd));
  OutStage od, oy;
  if (D) TRY(stage_out(h, "D", D, mb, &od));
  if (K > 0) TRY(stage_out(h, "Y", D1, (size_t)K * mb, &oy));
  const int64_t np = pad_n(N, o.mode);
  Ctx c;
  TRY(make_ctx(h, o.mode, N, np, o.time_kernels != 0, &c));
  MatBuf X[2], Y[2];
  Sp2Out r;
  TRY(run_sp2(h, Hd, N, dtype, nocc, o, Bd, K, h1_diag_only, false, X, Y, c, &r));
  if (D) {
    CK(launch_copy_out(r.xout, N, np, 1, o.mode, 1.0, od.dev, dtype, h->stream));
    c.kernels++;
    TRY(finish_out(h, od));
  }
  if (K > 0) {
    CK(launch_copy_out(r.yout, N, np, K, o.mode, 1.0, oy.dev, dtype, h->stream));
    c.kernels++;
    TRY(finish_out(h, oy));
  }
  auto* p = new sp2_handle_s::Pending();
  p->sp2 = true;
  p->r = r;
  p->c = c;
  if (!r.converged) {
    p->status = SP2_ENOCONV;
    p->msg = "no convergence in " + std::to_string(r.M) + " steps";
  }
  return finish_call(h, p, info, (D && od.host) || (K > 0 && oy.host));
}

int sp2_adjoint(sp2_handle_t h, const void* G, int64_t N, int dtype, void* grad, sp2_info* info);

int sp2_susceptibility(sp2_handle_t h, const void* H, int64_t N, int dtype, double nocc,
                       const void* A, int64_t L, int a_diag_only, int direction,
                       const sp2_opts* opts_in, void* D, void* chi, sp2_info* info) {
  TRY(check_common(h, H, N, dtype, nocc));
  if (L < 0) return fail(h, SP2_EINVAL, "L < 0");
  if (direction != 0 && direction != 1) return fail(h, SP2_EINVAL, "direction must be 0 or 1");
  if (N > 0 && L > 0 && (!A || !chi)) return fail(h, SP2_EINVAL, "A or chi is NULL");
  sp2_opts o = resolve(opts_in);
  TRY(validate_opts(h, &o));
  if (direction == 0)
    return sp2_response(h, H, N, dtype, nocc, A, L, a_diag_only, &o, D, chi, info);
  if (info) memset(info, 0, sizeof *info);
  if (N == 0) {
    if (info) info->converged = 1;
    return SP2_OK;
  }
  // backward: forward pass with checkpoints, then Eq. DM2
  const size_t mb = (size_t)N * N * dsize(dtype);
  const size_t b_bytes = (size_t)L * (a_diag_only ? N : N * N) * dsize(dtype);
  const void *Hd, *Bd = nullptr;
  TRY(stage_in(h, "H", H, mb, &Hd));
  if (L > 0) TRY(stage_in(h, "B", A, b_bytes, &Bd));
  OutStage od, oy;
  if (D) TRY(stage_out(h, "D", D, mb, &od));
  if (L > 0) TRY(stage_out(h, "Y", chi, (size_t)L * mb, &oy));
  const int64_t np = pad_n(N, o.mode);
  Ctx c;
  TRY(make_ctx(h, o.mode, N, np, o.time_kernels != 0, &c));
  MatBuf X[2], Y[2];
  Sp2Out r;
  h->hist.valid = false;
  TRY(resolve_ckpt(h, &o, np, L));
  TRY(run_sp2(h, Hd, N, dtype, nocc, o, nullptr, 0, 0, true, X, Y, c, &r));
  if (D) {
    CK(launch_copy_out(r.xout, N, np, 1, o.mode, 1.0, od.dev, dtype, h->stream));
    c.kernels++;
    // D is final before the adjoint starts: a host copy of it runs beside the adjoint
    TRY(finish_out_beside(h, od));
  }
  TRY(keep_history(h, r, N, np, o.mode, o.ckpt_k, c.tail));
  auto* p = new sp2_handle_s::Pending();
  if (L > 0) {
    TRY(run_adjoint(h, Bd, L, a_diag_only, 0, dtype, oy.dev, dtype, c, &p->adj_state));
    TRY(finish_out(h, oy));
  }
  TRY(join_beside(h));
  p->sp2 = true;
  p->r = r;
  p->c = c;
  p->ckpt_k = o.ckpt_k;
  p->hist_sigma = true;
  if (!r.converged) {
    p->status = SP2_ENOCONV;
    p->msg = "no convergence in " + std::to_string(r.M) + " steps";
  }
  return finish_call(h, p, info, (D && od.host) || (L > 0 && oy.host));
}

int sp2_adjoint(sp2_handle_t h, const void* G, int64_t N, int dtype, void* grad, sp2_info* info) {
  if (!h) return SP2_EINVAL;
  if (!h->hist.valid) return fail(h, SP2_ENOSTATE, "no X_n history kept on this handle");
  if (N != h->hist.n) return fail(h, SP2_ENOSTATE, "N = %lld differs from the kept history (%lld)",
                                  (long long)N, (long long)h->hist.n);
  if (dtype != SP2_F64 && dtype != SP2_F32) return fail(h, SP2_EINVAL, "unknown dtype %d", dtype);
  if (N == 0) return SP2_OK;
  if (!G || !grad) return fail(h, SP2_EINVAL, "G or grad is NULL");
  const size_t mb = (size_t)N * N * dsize(dtype);
  const void* Gd;
  TRY(stage_in(h, "B", G, mb, &Gd));
  OutStage oy;
  TRY(stage_out(h, "Y", grad, mb, &oy));
  Ctx c;
  TRY(make_ctx(h, h->hist.mode, h->hist.n, h->hist.np, true, &c));
  auto* p = new sp2_handle_s::Pending();
  p->adjoint = true;
  int code = run_adjoint(h, Gd, 1, 0, 1, dtype, oy.dev, dtype, c, &p->adj_state);
  if (code == SP2_OK) code = finish_out(h, oy);
  if (code != SP2_OK) {
    delete p;
    return code;
  }
  p->c = c;
  return finish_call(h, p, info, oy.host);
}

int sp2_release_history(sp2_handle_t h) {
  if (!h) return SP2_EINVAL;
  h->hist.valid = false;
  std::vector<std::string> names;
  for (auto& kv : h->bufs)
    if (kv.first.rfind("ckpt.", 0) == 0 || kv.first.rfind("seg.", 0) == 0) names.push_back(kv.first);
  cudaStreamSynchronize(h->stream);
  for (auto& nm : names) ws_free(h, nm);
  return SP2_OK;
}


}  // extern "C"

// --------------------------------------------------------------- finite temperature driver
namespace {

// The forward pass of the finite-temperature recursion (Sec. V.B, tanh doubling
// delta_{j+1} = 2 delta_j W_j, W_j = (I + 4 delta_j^2)^-1) with its history, kept
// for any number of responses; with `canonical`, also the response R_I to the
// identity and its trace, for mu_1 such that Tr[D1] = 0.
struct FermiState {
  int n = 0;                 // doublings
  double cst = 0.0;          // beta / 2^(n+2)
  double emin = 0.0, emax = 0.0;
  bool canonical = false;
  std::vector<FMat> dl, W;   // delta_0..delta_n, W_0..W_{n-1}
  FMat P, S, T, U, Z2[2];    // scratch of the forward pass and the responses
  FMat dd[2], E, F1, dW, G1, RI;
  double trI = 0.0;
  void* tr = nullptr;        // 2 device doubles
};

int fermi_response(Ctx& c, FermiState& fs, const void* src, int dtype, int diag, bool isI,
                   FMat** result);

int fermi_setup(Ctx& c, FermiState& fs, const void* Hd, int64_t N, int dtype, double mu, double kT,
                int n_doublings, bool canonical, bool responses) {
  sp2_handle_t h = c.h;
  const int mode = c.mode;
  const int64_t np = c.np;
  CK(cudaMemsetAsync(h->d_state, 0, sizeof(DevState), h->stream));  // never halted
  // spectral bound of H - mu I (Gershgorin, Sec. II estimates)
  const int nb = bounds_nparts(N);
  void* bp;
  TRY(ws(h, "bounds.part", nb * sizeof(double2), &bp));
  CK(launch_bounds(Hd, N, dtype, static_cast<double2*>(bp), nb, h->d_state, h->stream));
  c.kernels += 2;
  TRY(poll_state(h));
  fs.emin = h->h_state->bounds[0];
  fs.emax = h->h_state->bounds[1];
  if (!std::isfinite(fs.emin) || !std::isfinite(fs.emax))
    return fail(h, SP2_ENONFINITE, "non-finite spectral bounds (NaN/Inf in H)");
  fs.cst = 1.0 / (kT * std::ldexp(1.0, n_doublings + 2));
  double b = fs.cst * std::fmax(std::fabs(fs.emax - mu), std::fabs(fs.emin - mu));
  if (!(b < 0.5))
    return fail(h, SP2_EINVAL, "n_doublings = %d too small: |e - mu| / (kT 2^(n+2)) reaches %g >= 1/2",
                n_doublings, b);
  const double tol = mode == SP2_MODE_FP64 ? 1e-17 : 1e-8;
  const int n = n_doublings;
  fs.n = n;
  fs.canonical = canonical;
  fs.dl.assign(n + 1, FMat{});
  fs.W.assign(n, FMat{});
  for (int j = 0; j <= n; ++j) TRY(fmat(h, "ft.d" + std::to_string(j), np, mode, &fs.dl[j]));
  for (int j = 0; j < n; ++j) TRY(fmat(h, "ft.W" + std::to_string(j), np, mode, &fs.W[j]));
  TRY(fmat(h, "ft.P", np, mode, &fs.P));
  TRY(fmat(h, "ft.S", np, mode, &fs.S));
  TRY(fmat(h, "ft.T", np, mode, &fs.T));
  TRY(fmat(h, "ft.U", np, mode, &fs.U));
  TRY(fmat(h, "ft.Z0", np, mode, &fs.Z2[0]));
  TRY(fmat(h, "ft.Z1", np, mode, &fs.Z2[1]));
  // delta_0 = c mu I - c H (planes with scale 1: |delta| < 1/2)
  CK(launch_init(Hd, N, np, 1, dtype, 0, 0, fs.cst * mu, -fs.cst, mode, fs.dl[0].m, nullptr, 0,
                 nullptr, h->stream));
  c.kernels++;
  if (mode == SP2_MODE_FP16X2) {
    const float one = 1.0f;
    CK(cudaMemcpyAsync(fs.dl[0].scale, &one, sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  for (int j = 0; j < n; ++j) {
    // S = I + 4 delta^2, symmetrised: I + 2 (P + P^T)
    TRY(fprod(c, fs.P, fs.dl[j], fs.dl[j]));
    TRY(fcomb(c, fs.S, &fs.P, 2.0, nullptr, 0.0, nullptr, 0.0, 1.0, true));
    // W = S^{-1} by Newton-Schulz: Z <- 2 Z - sym(Z (S Z))
    const int kns = ns_iterations(b, tol);
    const double z0 = 2.0 / (2.0 + 4.0 * b * b);
    int zi = 0;
    FMat* Zc = (kns == 0) ? &fs.W[j] : &fs.Z2[0];
    TRY(fcomb(c, *Zc, nullptr, 0.0, nullptr, 0.0, nullptr, 0.0, z0, true));
    for (int it = 0; it < kns; ++it) {
      FMat& Zin = *Zc;
      FMat& Zout = (it == kns - 1) ? fs.W[j] : fs.Z2[1 - zi];
      TRY(fprod(c, fs.T, fs.S, Zin));
      TRY(fplanes(c, fs.T));
      TRY(fprod(c, fs.U, Zin, fs.T));
      TRY(fcomb(c, Zout, &fs.U, -0.5, nullptr, 0.0, &Zin, 2.0, 0.0, true));
      zi = 1 - zi;
      Zc = &Zout;
    }
    // delta_{j+1} = 2 delta W, symmetrised: V + V^T with V = delta W
    TRY(fprod(c, fs.P, fs.dl[j], fs.W[j]));
    TRY(fcomb(c, fs.dl[j + 1], &fs.P, 1.0, nullptr, 0.0, nullptr, 0.0, 0.0, true));
    b = 2.0 * b / (1.0 + 4.0 * b * b);
  }
  if (!responses) return SP2_OK;
  TRY(fmat(h, "ft.dd0", np, mode, &fs.dd[0]));
  TRY(fmat(h, "ft.dd1", np, mode, &fs.dd[1]));
  TRY(fmat(h, "ft.E", np, mode, &fs.E));
  TRY(fmat(h, "ft.F1", np, mode, &fs.F1));
  TRY(fmat(h, "ft.dW", np, mode, &fs.dW));
  TRY(fmat(h, "ft.G1", np, mode, &fs.G1));
  TRY(ws(h, "ft.tr", 2 * sizeof(double), &fs.tr));
  if (canonical) {
    TRY(fmat(h, "ft.RI", np, mode, &fs.RI));
    void* ones = nullptr;
    TRY(ws(h, "ft.ones", (size_t)N * dsize(dtype), &ones));
    std::vector<double> h1(N, 1.0);
    std::vector<float> h1f(N, 1.0f);
    CK(cudaMemcpyAsync(ones, dtype == SP2_F64 ? (const void*)h1.data() : (const void*)h1f.data(),
                       (size_t)N * dsize(dtype), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    FMat* r;
    TRY(fermi_response(c, fs, ones, dtype, 1, true, &r));   // the response to I first
  }
  return SP2_OK;
}

// First-order response of f(H) to B (chain rule of every doubling); canonical
// adds -(Tr D1 / Tr R_I) R_I. *result points at the FMat holding it (scratch
// of fs, valid until the next response).
int fermi_response(Ctx& c, FermiState& fs, const void* src, int dtype, int diag, bool isI,
                   FMat** result) {
  sp2_handle_t h = c.h;
  const int mode = c.mode;
  const int n = fs.n;
  double* tr = static_cast<double*>(fs.tr);
  int cur = 0;
  FMat& d0 = fs.dd[0];
  if (mode == SP2_MODE_FP16X2) CK(cudaMemsetAsync(d0.amax, 0, sizeof(float), h->stream));
  CK(launch_init(src, c.n, c.np, 1, dtype, diag, 0, 0.0, -fs.cst, mode, d0.m, nullptr, 0,
                 mode == SP2_MODE_FP16X2 ? d0.amax : nullptr, h->stream));
  c.kernels++;
  if (mode == SP2_MODE_FP16X2) TRY(fplanes(c, d0));
  for (int j = 0; j < n; ++j) {
    FMat& din = fs.dd[cur];
    FMat& dout = (j == n - 1 && isI) ? fs.RI : fs.dd[1 - cur];
    // E = d delta delta + delta d delta = Z1 + Z1^T, Z1 = d delta * delta
    TRY(fprod(c, fs.P, din, fs.dl[j]));
    TRY(fcomb(c, fs.E, &fs.P, 1.0, nullptr, 0.0, nullptr, 0.0, 0.0, true));
    // dW = -4 W E W = -2 (F2 + F2^T), F2 = (W E) W
    TRY(fprod(c, fs.F1, fs.W[j], fs.E));
    TRY(fplanes(c, fs.F1));
    TRY(fprod(c, fs.U, fs.F1, fs.W[j]));
    TRY(fcomb(c, fs.dW, &fs.U, -2.0, nullptr, 0.0, nullptr, 0.0, 0.0, true));
    // d delta' = 2 (d delta W + delta dW) = (G1 + G1^T) + (G2 + G2^T)
    TRY(fprod(c, fs.G1, din, fs.W[j]));
    TRY(fprod(c, fs.T, fs.dl[j], fs.dW));
    TRY(fcomb(c, dout, &fs.G1, 1.0, &fs.T, 1.0, nullptr, 0.0, 0.0, j < n - 1));
    cur = 1 - cur;
  }
  if (isI) {
    CK(launch_trace(mode, fs.RI.m.master, c.np, c.n, tr + 1, h->stream));
    CK(cudaMemcpyAsync(&h->h_state->bounds[1], tr + 1, sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    fs.trI = h->h_state->bounds[1];
    c.kernels++;
    *result = &fs.RI;
    return SP2_OK;
  }
  FMat& res = fs.dd[cur];
  *result = &res;
  if (fs.canonical) {
    CK(launch_trace(mode, res.m.master, c.np, c.n, tr, h->stream));
    CK(cudaMemcpyAsync(&h->h_state->bounds[0], tr, sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const double trk = h->h_state->bounds[0];
    c.kernels++;
    // res - (trk / trI) RI, written as (a/2)(RI + RI^T) + res (RI is exactly symmetric)
    TRY(fcomb(c, fs.G1, &fs.RI, -0.5 * trk / fs.trI, nullptr, 0.0, &res, 1.0, 0.0, false));
    *result = &fs.G1;
  }
  return SP2_OK;
}

}  // namespace

extern "C" {

int sp2_fermi(sp2_handle_t h, const void* H, int64_t N, int dtype, double mu, double kT,
              const void* B, int64_t K, int b_diag_only, int canonical, int n_doublings,
              const sp2_opts* opts_in, void* D, void* D1, sp2_info* info) {
  if (h) drop_pending(h);   // this call completes before it returns
  if (!h) return SP2_EINVAL;
  if (N < 0 || K < 0) return fail(h, SP2_EINVAL, "negative size");
  if (dtype != SP2_F64 && dtype != SP2_F32) return fail(h, SP2_EINVAL, "unknown dtype %d", dtype);
  if (!(kT > 0.0) || !std::isfinite(mu)) return fail(h, SP2_EINVAL, "kT must be > 0, mu finite");
  if (n_doublings < 1 || n_doublings > 64) return fail(h, SP2_EINVAL, "n_doublings outside 1..64");
  if (N > 0 && (!H || (K > 0 && (!B || !D1)))) return fail(h, SP2_EINVAL, "null pointer");
  sp2_opts o = resolve(opts_in);
  TRY(validate_opts(h, &o));
  if (o.block_sparse) return fail(h, SP2_EINVAL, "block_sparse: sp2_density only");
  if (info) memset(info, 0, sizeof *info);
  if (N == 0) {
    if (info) info->converged = 1;
    return SP2_OK;
  }
  const int mode = o.mode;
  const int64_t np = pad_n(N, mode);
  const size_t mb = (size_t)N * N * dsize(dtype);
  const void *Hd, *Bd = nullptr;
  TRY(stage_in(h, "H", H, mb, &Hd));
  if (K > 0) TRY(stage_in(h, "B", B, (size_t)K * (b_diag_only ? N : N * N) * dsize(dtype), &Bd));
  OutStage od, oy;
  if (D) TRY(stage_out(h, "D", D, mb, &od));
  if (K > 0) TRY(stage_out(h, "Y", D1, (size_t)K * mb, &oy));
  Ctx c;
  TRY(make_ctx(h, mode, N, np, o.time_kernels != 0, &c));
  FermiState fs;
  TRY(fermi_setup(c, fs, Hd, N, dtype, mu, kT, n_doublings, canonical != 0, K > 0));
  // D = I/2 + delta_n
  if (D) {
    TRY(fcomb(c, fs.P, nullptr, 0.0, nullptr, 0.0, &fs.dl[fs.n], 1.0, 0.5, false));
    CK(launch_copy_out(fs.P.m, N, np, 1, mode, 1.0, od.dev, dtype, h->stream));
    c.kernels++;
    TRY(finish_out(h, od));
  }
  const int64_t per = b_diag_only ? N : N * N;
  for (int64_t kk = K - 1; kk >= 0; --kk) {
    FMat* r;
    TRY(fermi_response(c, fs, static_cast<const char*>(Bd) + (size_t)kk * per * dsize(dtype), dtype,
                       b_diag_only, false, &r));
    CK(launch_copy_out(r->m, N, np, 1, mode, 1.0,
                       static_cast<char*>(oy.dev) + (size_t)kk * N * N * dsize(dtype), dtype,
                       h->stream));
    c.kernels++;
  }
  if (K > 0) TRY(finish_out(h, oy));
  CK(cudaStreamSynchronize(h->stream));
  if (info) {
    info->M = fs.n;
    info->converged = 1;
    info->alpha = 0.5;
    info->beta = -fs.cst;
    info->eps_min = fs.emin;
    info->eps_max = fs.emax;
  }
  fill_timing(c, 1 << 30, info);
  return SP2_OK;
}

}  // extern "C"

// --------------------------------------------------------------- non-orthonormal basis
namespace {

// caller matrix (N x N, dtype) -> padded FMat times `scale`, with planes
int fload(Ctx& c, FMat& f, const void* src, int dtype, double scale) {
  sp2_handle_t h = c.h;
  const bool f16 = c.mode == SP2_MODE_FP16X2;
  if (f16) CK(cudaMemsetAsync(f.amax, 0, sizeof(float), h->stream));
  CK(launch_init(src, c.n, c.np, 1, dtype, 0, 1, 0.0, scale, c.mode, f.m, nullptr, 0,
                 f16 ? f.amax : nullptr, h->stream));
  c.kernels++;
  if (f16) TRY(fplanes(c, f));
  return SP2_OK;
}

// C = sym(L M R) for symmetric R: the middle product's planes are formed for its
// use as the row operand of the second product (scratch T1, T2)
int fsandwich(Ctx& c, FMat& C, const FMat& L, const FMat& Mid, const FMat& R, FMat& T1, FMat& T2) {
  TRY(fprod(c, T1, L, Mid));
  TRY(fplanes(c, T1));
  TRY(fprod(c, T2, T1, R));
  return fcomb(c, C, &T2, 0.5, nullptr, 0.0, nullptr, 0.0, 0.0, true);
}

// ||T - I||_F^2 of the padded master (zero outside the caller's block), FP64
int dist_to_identity(Ctx& c, const FMat& T, double* out) {
  sp2_handle_t h = c.h;
  void* p;
  TRY(ws(h, "no.red", 4 * sizeof(double), &p));
  double* d = static_cast<double*>(p);
  const int mdt = c.mode == SP2_MODE_FP64 ? SP2_F64 : SP2_F32;
  const int np_ = contract_nparts(c.np, 0);
  void* part;
  TRY(ws(h, "no.part", (size_t)np_ * sizeof(double), &part));
  CK(launch_contract(T.m.master, 1, T.m.master, 1, c.np, mdt, 0, static_cast<double*>(part), np_,
                     d, h->stream));
  CK(launch_trace(c.mode, T.m.master, c.np, c.n, d + 1, h->stream));
  double hv[2];
  CK(cudaMemcpyAsync(hv, d, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  c.kernels += 2;
  *out = hv[0] - 2.0 * hv[1] + (double)c.n;
  return SP2_OK;
}

}  // namespace

extern "C" {

int sp2_nonorth_susceptibility(sp2_handle_t h, const void* H, const void* S, int64_t N, int dtype,
                               double nocc, const void* A, const sp2_opts* opts_in, void* D,
                               void* WH, void* WS, void* Zout, sp2_info* info) {
  if (h) drop_pending(h);   // this call completes before it returns
  TRY(check_common(h, H, N, dtype, nocc));
  if (N > 0 && (!S || !A || !D || !WH || !WS)) return fail(h, SP2_EINVAL, "null pointer");
  sp2_opts o = resolve(opts_in);
  TRY(validate_opts(h, &o));
  if (o.block_sparse) return fail(h, SP2_EINVAL, "block_sparse: sp2_density only");
  if (o.fixed_m > 0) return fail(h, SP2_EINVAL, "fixed_m is not supported here");
  if (info) memset(info, 0, sizeof *info);
  if (N == 0) {
    if (info) info->converged = 1;
    return SP2_OK;
  }
  const int mode = o.mode;
  const int64_t np = pad_n(N, mode);
  const size_t mb = (size_t)N * N * dsize(dtype);
  const void *Hd, *Sd, *Ad;
  TRY(stage_in(h, "H", H, mb, &Hd));
  TRY(stage_in(h, "no.S", S, mb, &Sd));
  TRY(stage_in(h, "B", A, mb, &Ad));
  OutStage od, oh, os, oz;
  TRY(stage_out(h, "no.D", D, mb, &od));
  TRY(stage_out(h, "no.WH", WH, mb, &oh));
  TRY(stage_out(h, "no.WS", WS, mb, &os));
  if (Zout) TRY(stage_out(h, "no.Z", Zout, mb, &oz));
  Ctx c;
  TRY(make_ctx(h, mode, N, np, o.time_kernels != 0, &c));
  CK(cudaMemsetAsync(h->d_state, 0, sizeof(DevState), h->stream));

  // Loewdin factor Z = S^(-1/2) by the coupled Newton-Schulz iteration on S / s0,
  // s0 the Gershgorin upper bound of S (spectrum of S / s0 in (0, 1]):
  //   T = (3 I - Zk Yk) / 2,  Yk <- Yk T -> (S/s0)^(1/2),  Zk <- T Zk -> (S/s0)^(-1/2).
  // Every iterate is a polynomial in S, so all factors commute and are symmetric.
  const int nb = bounds_nparts(N);
  void* bp;
  TRY(ws(h, "bounds.part", nb * sizeof(double2), &bp));
  CK(launch_bounds(Sd, N, dtype, static_cast<double2*>(bp), nb, h->d_state, h->stream));
  c.kernels += 2;
  TRY(poll_state(h));
  const double s0 = h->h_state->bounds[1];
  if (!std::isfinite(s0) || !(s0 > 0.0))
    return fail(h, SP2_EINVAL, "overlap matrix with non-positive or non-finite Gershgorin bound");
  FMat Y, Zk, T, P, Q, Q2, Z, Sinv, Hm, Am, Hp, Ap, Dp, Cp, Dm, Wh, Ws;
  TRY(fmat(h, "no.Y", np, mode, &Y));
  TRY(fmat(h, "no.Zk", np, mode, &Zk));
  TRY(fmat(h, "no.T", np, mode, &T));
  TRY(fmat(h, "no.P", np, mode, &P));
  TRY(fmat(h, "no.Q", np, mode, &Q));
  TRY(fmat(h, "no.Q2", np, mode, &Q2));
  TRY(fload(c, Y, Sd, dtype, 1.0 / s0));
  TRY(fcomb(c, Zk, nullptr, 0.0, nullptr, 0.0, nullptr, 0.0, 1.0, true));
  const double tol = mode == SP2_MODE_FP64 ? 1e-26 * (double)N : 1e-12 * (double)N;
  double prev = 0.0;
  int its = 0, stall = 0;
  for (; its < 100; ++its) {
    TRY(fprod(c, P, Zk, Y));
    TRY(fcomb(c, T, &P, -0.25, nullptr, 0.0, nullptr, 0.0, 1.5, true));
    double e;
    TRY(dist_to_identity(c, T, &e));  // ||T - I||^2 = ||I - Zk Yk||^2 / 4
    if (!std::isfinite(e)) return fail(h, SP2_ENONFINITE, "non-finite Newton-Schulz residual");
    if (e <= tol) break;
    // below 1e-6 an iteration that does not halve the residual has reached the
    // rounding floor of the mode (twice in a row ends the iteration)
    if (its > 0 && e < 1e-6 * (double)N && e > 0.25 * prev) {
      if (++stall >= 2) break;
    } else {
      stall = 0;
    }
    prev = e;
    TRY(fprod(c, Q, Y, T));
    TRY(fprod(c, Q2, T, Zk));
    TRY(fcomb(c, Y, &Q, 0.5, nullptr, 0.0, nullptr, 0.0, 0.0, true));
    TRY(fcomb(c, Zk, &Q2, 0.5, nullptr, 0.0, nullptr, 0.0, 0.0, true));
  }
  if (its >= 100) return fail(h, SP2_ENOCONV, "inverse square root of S did not converge");
  TRY(fmat(h, "no.Z", np, mode, &Z));
  TRY(fmat(h, "no.Sinv", np, mode, &Sinv));
  TRY(fcomb(c, Z, &Zk, 0.5 / std::sqrt(s0), nullptr, 0.0, nullptr, 0.0, 0.0, true));
  TRY(fprod(c, Q, Z, Z));
  TRY(fcomb(c, Sinv, &Q, 0.5, nullptr, 0.0, nullptr, 0.0, 0.0, true));  // S^(-1) = Z Z

  // orthonormalised H and A (Sec. V.A congruences)
  TRY(fmat(h, "no.H", np, mode, &Hm));
  TRY(fmat(h, "no.A", np, mode, &Am));
  TRY(fmat(h, "no.Hp", np, mode, &Hp));
  TRY(fmat(h, "no.Ap", np, mode, &Ap));
  TRY(fload(c, Hm, Hd, dtype, 1.0));
  TRY(fload(c, Am, Ad, dtype, 1.0));
  TRY(fsandwich(c, Hp, Z, Hm, Z, P, Q));
  TRY(fsandwich(c, Ap, Z, Am, Z, P, Q));

  // D^perp and chi^(A^perp): the SP2 density and the backward susceptibility (Eq. DM2)
  const int idt = mode == SP2_MODE_FP64 ? SP2_F64 : SP2_F32;
  const size_t ib = (size_t)N * N * dsize(idt);
  void *hpn, *apn, *dpn, *cpn;
  TRY(ws(h, "no.Hpn", ib, &hpn));
  TRY(ws(h, "no.Apn", ib, &apn));
  TRY(ws(h, "no.Dpn", ib, &dpn));
  TRY(ws(h, "no.Cpn", ib, &cpn));
  CK(launch_copy_out(Hp.m, N, np, 1, mode, 1.0, hpn, idt, h->stream));
  CK(launch_copy_out(Ap.m, N, np, 1, mode, 1.0, apn, idt, h->stream));
  c.kernels += 2;
  const int64_t k0 = c.kernels, l0 = c.launches;
  const double f0 = c.flops, a0 = c.alg;
  sp2_info si;
  TRY(sp2_susceptibility(h, hpn, N, idt, nocc, apn, 1, 0, 1, &o, dpn, cpn, &si));
  TRY(make_ctx(h, mode, N, np, o.time_kernels != 0, &c));  // fresh partials after the solve
  c.kernels = k0 + si.kernel_launches;
  c.launches = l0 + si.n_gemm_launches;
  c.flops = f0 + si.executed_flops;
  c.alg = a0 + si.algorithmic_flops;
  c.st = h->d_state;
  CK(cudaMemsetAsync(h->d_state, 0, sizeof(DevState), h->stream));

  // back to the atomic-orbital representation and the dual weights:
  //   D = Z D^perp Z,  W_H = Z chi^perp Z,  W_S = -sym(S^-1 H W_H) - sym(S^-1 A D)
  TRY(fmat(h, "no.Dp", np, mode, &Dp));
  TRY(fmat(h, "no.Cp", np, mode, &Cp));
  TRY(fmat(h, "no.Dm", np, mode, &Dm));
  TRY(fmat(h, "no.Wh", np, mode, &Wh));
  TRY(fmat(h, "no.Ws", np, mode, &Ws));
  TRY(fload(c, Dp, dpn, idt, 1.0));
  TRY(fload(c, Cp, cpn, idt, 1.0));
  TRY(fsandwich(c, Dm, Z, Dp, Z, P, Q));
  TRY(fsandwich(c, Wh, Z, Cp, Z, P, Q));
  TRY(fprod(c, P, Sinv, Hm));
  TRY(fplanes(c, P));
  TRY(fprod(c, Q, P, Wh));           // M = S^-1 H W_H
  TRY(fprod(c, P, Sinv, Am));
  TRY(fplanes(c, P));
  TRY(fprod(c, Q2, P, Dm));          // S^-1 A D
  TRY(fcomb(c, Ws, &Q, -0.5, &Q2, -0.5, nullptr, 0.0, 0.0, false));
  CK(launch_copy_out(Dm.m, N, np, 1, mode, 1.0, od.dev, dtype, h->stream));
  CK(launch_copy_out(Wh.m, N, np, 1, mode, 1.0, oh.dev, dtype, h->stream));
  CK(launch_copy_out(Ws.m, N, np, 1, mode, 1.0, os.dev, dtype, h->stream));
  c.kernels += 3;
  if (Zout) {
    CK(launch_copy_out(Z.m, N, np, 1, mode, 1.0, oz.dev, dtype, h->stream));
    c.kernels++;
    TRY(finish_out(h, oz));
  }
  TRY(finish_out(h, od));
  TRY(finish_out(h, oh));
  TRY(finish_out(h, os));
  CK(cudaStreamSynchronize(h->stream));
  if (info) {
    *info = si;
    info->n_gemm_launches = c.launches;
    info->executed_flops = c.flops;
    info->algorithmic_flops = c.alg;
    info->kernel_launches = c.kernels;
    info->refine_iter = its;   // Newton-Schulz iterations of the inverse square root
  }
  return SP2_OK;
}

int response_contract(sp2_handle_t h, const void* P, int64_t L, const void* Q, int64_t K, int64_t N,
                      int dtype, int q_diag_only, double* out) {
  if (!h) return SP2_EINVAL;
  if (L < 0 || K < 0 || N < 0) return fail(h, SP2_EINVAL, "negative size");
  if (dtype != SP2_F64 && dtype != SP2_F32) return fail(h, SP2_EINVAL, "unknown dtype %d", dtype);
  if (L == 0 || K == 0) return SP2_OK;
  if (!out) return fail(h, SP2_EINVAL, "out is NULL");
  if (N == 0) {
    OutStage oo;
    TRY(stage_out(h, "out", out, (size_t)L * K * sizeof(double), &oo));
    CK(cudaMemsetAsync(oo.dev, 0, (size_t)L * K * sizeof(double), h->stream));
    TRY(finish_out(h, oo));
    CK(cudaStreamSynchronize(h->stream));
    return SP2_OK;
  }
  if (!P || !Q) return fail(h, SP2_EINVAL, "P or Q is NULL");
  const void *Pd, *Qd;
  TRY(stage_in(h, "P", P, (size_t)L * N * N * dsize(dtype), &Pd));
  TRY(stage_in(h, "Q", Q, (size_t)K * (q_diag_only ? N : N * N) * dsize(dtype), &Qd));
  OutStage oo;
  TRY(stage_out(h, "out", out, (size_t)L * K * sizeof(double), &oo));
  int np_ = contract_nparts(N, q_diag_only);
  if (L * K >= 8 && np_ > 304) np_ = 304;   // many pairs already fill the GPU
  if ((int64_t)np_ * L * K > (int64_t)1 << 24) {   // partials of many pairs: at most 128 MiB
    const int64_t m = ((int64_t)1 << 24) / (L * K);
    np_ = (int)(m < 1 ? 1 : m);
  }
  void* part;
  TRY(ws(h, "contract.part", (size_t)L * K * np_ * sizeof(double), &part));
  CK(launch_contract(Pd, L, Qd, K, N, dtype, q_diag_only, static_cast<double*>(part), np_,
                     static_cast<double*>(oo.dev), h->stream));
  TRY(finish_out(h, oo));
  CK(cudaStreamSynchronize(h->stream));
  return SP2_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- SCF response + MLP
namespace {

// Solve the (m+1) x (m+1) Anderson system [G 1; 1^T 0] [c; lam] = [0; 1]
// by Gaussian elimination with partial pivoting (host, tiny). G gets a
// relative Tikhonov shift for rank-deficient histories.
void anderson_coeffs(const double* G, int m, double* c) {
  double A[33][34];
  double tr = 0.0;
  for (int i = 0; i < m; ++i) tr += G[i * m + i];
  const double shift = 1e-12 * (tr > 0 ? tr / m : 1.0);
  for (int i = 0; i <= m; ++i)
    for (int j = 0; j <= m + 1; ++j) A[i][j] = 0.0;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) A[i][j] = G[i * m + j];
    A[i][i] += shift;
    A[i][m] = 1.0;
    A[m][i] = 1.0;
  }
  A[m][m + 1] = 1.0;
  const int n = m + 1;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i][k]) > std::fabs(A[p][k])) p = i;
    if (p != k)
      for (int j = 0; j <= n; ++j) std::swap(A[k][j], A[p][j]);
    const double d = A[k][k];
    if (d == 0.0) continue;
    for (int i = k + 1; i < n; ++i) {
      const double f = A[i][k] / d;
      for (int j = k; j <= n; ++j) A[i][j] -= f * A[k][j];
    }
  }
  double x[33];
  for (int i = n - 1; i >= 0; --i) {
    double s = A[i][n];
    for (int j = i + 1; j < n; ++j) s -= A[i][j] * x[j];
    x[i] = A[i][i] != 0.0 ? s / A[i][i] : 0.0;
  }
  for (int i = 0; i < m; ++i) c[i] = x[i];
}

// MLP forward for a batch: Hr = relu(X W1^T) (P x dh), Y = Hr W2^T (P x din)
int mlp_fwd(sp2_handle_t h, const float* W1, const float* W2, int din, int dh, const float* X,
            int64_t P, float* Hr, float* Y, int bf16) {
  CK(launch_sgemm(P, dh, din, 1.0f, X, din, 0, W1, din, 1, 0.0f, Hr, dh, 1, bf16, h->stream));
  CK(launch_sgemm(P, din, dh, 1.0f, Hr, dh, 0, W2, dh, 1, 0.0f, Y, din, 0, bf16, h->stream));
  return SP2_OK;
}

// loss and gradients (backpropagation through y = W2 relu(W1 x)); loss on device
int mlp_grad(sp2_handle_t h, const float* W1, const float* W2, int din, int dh, const float* X,
             const float* T, int64_t P, double* dloss, float* dW1, float* dW2, float* Hr, float* Y,
             float* dY, float* dH) {
  TRY(mlp_fwd(h, W1, W2, din, dh, X, P, Hr, Y, 0));
  CK(cudaMemsetAsync(dloss, 0, sizeof(double), h->stream));
  CK(launch_mse_grad(Y, T, P * din, 1.0f / (float)P, dY, dloss, h->stream));
  // dW2 = dY^T Hr (din x dh); dH = dY W2 (P x dh) masked; dW1 = dH^T X (dh x din)
  CK(launch_sgemm(din, dh, P, 1.0f, dY, din, 1, Hr, dh, 0, 0.0f, dW2, dh, 0, 0, h->stream));
  CK(launch_sgemm(P, dh, din, 1.0f, dY, din, 0, W2, dh, 0, 0.0f, dH, dh, 0, 0, h->stream));
  CK(launch_relu_mask(dH, Hr, P * dh, h->stream));
  CK(launch_sgemm(dh, din, P, 1.0f, dH, dh, 1, X, din, 0, 0.0f, dW1, din, 0, 0, h->stream));
  return SP2_OK;
}

int mlp_scratch(sp2_handle_t h, int din, int dh, int64_t P, float** Hr, float** Y, float** dY,
                float** dH) {
  void *a, *b, *c2, *d;
  TRY(ws(h, "mlp.H", (size_t)P * dh * sizeof(float), &a));
  TRY(ws(h, "mlp.Y", (size_t)P * din * sizeof(float), &b));
  TRY(ws(h, "mlp.dY", (size_t)P * din * sizeof(float), &c2));
  TRY(ws(h, "mlp.dH", (size_t)P * dh * sizeof(float), &d));
  *Hr = static_cast<float*>(a);
  *Y = static_cast<float*>(b);
  *dY = static_cast<float*>(c2);
  *dH = static_cast<float*>(d);
  return SP2_OK;
}

}  // namespace

extern "C" {

int sp2_mlp_forward(sp2_handle_t h, const float* W1, const float* W2, int din, int dh,
                    const float* X, int64_t P, float* Y, int bf16) {
  if (!h) return SP2_EINVAL;
  if (din <= 0 || dh <= 0 || P < 0) return fail(h, SP2_EINVAL, "bad MLP sizes");
  if (P == 0) return SP2_OK;
  if (!W1 || !W2 || !X || !Y) return fail(h, SP2_EINVAL, "null pointer");
  void* a;
  TRY(ws(h, "mlp.H", (size_t)P * dh * sizeof(float), &a));
  TRY(mlp_fwd(h, W1, W2, din, dh, X, P, static_cast<float*>(a), Y, bf16));
  CK(cudaStreamSynchronize(h->stream));
  return SP2_OK;
}

int sp2_mlp_loss_grad(sp2_handle_t h, const float* W1, const float* W2, int din, int dh,
                      const float* X, const float* T, int64_t P, double* loss, float* dW1,
                      float* dW2) {
  if (!h) return SP2_EINVAL;
  if (din <= 0 || dh <= 0 || P <= 0) return fail(h, SP2_EINVAL, "bad MLP sizes");
  if (!W1 || !W2 || !X || !T || !dW1 || !dW2 || !loss) return fail(h, SP2_EINVAL, "null pointer");
  float *Hr, *Y, *dY, *dH;
  TRY(mlp_scratch(h, din, dh, P, &Hr, &Y, &dY, &dH));
  void* dl;
  TRY(ws(h, "mlp.loss", sizeof(double), &dl));
  TRY(mlp_grad(h, W1, W2, din, dh, X, T, P, static_cast<double*>(dl), dW1, dW2, Hr, Y, dY, dH));
  CK(cudaMemcpyAsync(loss, dl, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SP2_OK;
}

int sp2_mlp_train(sp2_handle_t h, float* W1, float* W2, int din, int dh, const float* X,
                  const float* T, int64_t P, int steps, double lr, double* loss_hist) {
  if (!h) return SP2_EINVAL;
  if (din <= 0 || dh <= 0 || P <= 0 || steps < 0) return fail(h, SP2_EINVAL, "bad MLP sizes");
  if (!W1 || !W2 || !X || !T) return fail(h, SP2_EINVAL, "null pointer");
  float *Hr, *Y, *dY, *dH;
  TRY(mlp_scratch(h, din, dh, P, &Hr, &Y, &dY, &dH));
  const int64_t n1 = (int64_t)dh * din, n2 = (int64_t)din * dh;
  void *g, *mv, *dl;
  TRY(ws(h, "mlp.g", (size_t)(n1 + n2) * sizeof(float), &g));
  TRY(ws(h, "mlp.mv", (size_t)2 * (n1 + n2) * sizeof(float), &mv));
  TRY(ws(h, "mlp.lossv", (size_t)(steps > 0 ? steps : 1) * sizeof(double), &dl));
  float* g1 = static_cast<float*>(g);
  float* g2 = g1 + n1;
  float* m1 = static_cast<float*>(mv);
  float* v1 = m1 + n1;
  float* m2 = v1 + n1;
  float* v2 = m2 + n2;
  CK(cudaMemsetAsync(mv, 0, (size_t)2 * (n1 + n2) * sizeof(float), h->stream));
  double* dloss = static_cast<double*>(dl);
  for (int t = 1; t <= steps; ++t) {
    TRY(mlp_grad(h, W1, W2, din, dh, X, T, P, dloss + (t - 1), g1, g2, Hr, Y, dY, dH));
    CK(launch_adam(W1, g1, m1, v1, n1, (float)lr, 0.9f, 0.999f, 1e-8f, t, h->stream));
    CK(launch_adam(W2, g2, m2, v2, n2, (float)lr, 0.9f, 0.999f, 1e-8f, t, h->stream));
  }
  if (loss_hist && steps > 0)
    CK(cudaMemcpyAsync(loss_hist, dloss, (size_t)steps * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SP2_OK;
}

int sp2_scf_response(sp2_handle_t h, const void* H, int64_t N, int dtype, double nocc, int norb,
                     const double* Ksite, const double* Vext, int64_t F, const sp2_scf_opts* so,
                     const sp2_opts* opts_in, double* q_out, double* residuals, int* iterations,
                     double* traj_r, double* traj_q, sp2_info* info) {
  if (h) drop_pending(h);   // this call completes before it returns
  TRY(check_common(h, H, N, dtype, nocc));
  if (!so) return fail(h, SP2_EINVAL, "null sp2_scf_opts");
  if (norb < 1 || N % norb != 0) return fail(h, SP2_EINVAL, "N must be a multiple of norb");
  if (F < 1 || !Ksite || !Vext || !q_out) return fail(h, SP2_EINVAL, "bad SCF arguments");
  if (so->max_iter < 1) return fail(h, SP2_EINVAL, "max_iter < 1");
  const bool anderson = so->mixer == SP2_MIX_ANDERSON || so->mixer == SP2_MIX_ANDERSON_MLP;
  const bool learned = so->mixer == SP2_MIX_MLP || so->mixer == SP2_MIX_ANDERSON_MLP;
  if (anderson && (so->history < 1 || so->history > 32))
    return fail(h, SP2_EINVAL, "Anderson history outside 1..32");
  if (learned && (!so->W1 || !so->W2 || so->hidden < 1))
    return fail(h, SP2_EINVAL, "MLP mixer needs W1, W2 and hidden");
  if (so->mixer < 0 || so->mixer > 3) return fail(h, SP2_EINVAL, "unknown mixer");
  const bool finite_t = so->kT > 0.0;
  const int ndbl = so->n_doublings > 0 ? so->n_doublings : 20;
  if (finite_t && (!std::isfinite(so->mu) || ndbl > 64))
    return fail(h, SP2_EINVAL, "finite-T SCF: mu must be finite, n_doublings <= 64");
  sp2_opts o = resolve(opts_in);
  TRY(validate_opts(h, &o));
  if (o.block_sparse) return fail(h, SP2_EINVAL, "block_sparse: sp2_density only");
  const bool refine = so->refine_below > 0.0 && so->refine_mode != o.mode;
  if (refine && so->refine_mode != SP2_MODE_FP64 && so->refine_mode != SP2_MODE_FP32 &&
      so->refine_mode != SP2_MODE_BF16X2 && so->refine_mode != SP2_MODE_FP16X2 &&
      so->refine_mode != SP2_MODE_BF16X3)
    return fail(h, SP2_EINVAL, "unknown refine_mode %d", so->refine_mode);
  if (info) memset(info, 0, sizeof *info);
  // one padding for every mode the loop may switch to (the split modes' 256)
  const int64_t ns = N / norb, np = pad_n(N, SP2_MODE_FP16X2), tot = F * ns;
  const size_t mb = (size_t)N * N * dsize(dtype);
  const void *Hd, *Kd, *Vd;
  TRY(stage_in(h, "H", H, mb, &Hd));
  TRY(stage_in(h, "scf.K", Ksite, (size_t)ns * ns * sizeof(double), &Kd));
  TRY(stage_in(h, "scf.V", Vext, (size_t)tot * sizeof(double), &Vd));
  OutStage oq;
  TRY(stage_out(h, "scf.qout", q_out, (size_t)tot * sizeof(double), &oq));
  void *pq, *pqo, *pr, *pu, *pub, *pn;
  TRY(ws(h, "scf.q", tot * sizeof(double), &pq));
  TRY(ws(h, "scf.qo", tot * sizeof(double), &pqo));
  TRY(ws(h, "scf.r", tot * sizeof(double), &pr));
  TRY(ws(h, "scf.u", tot * sizeof(double), &pu));
  TRY(ws(h, "scf.ub", (size_t)F * N * dsize(dtype), &pub));
  TRY(ws(h, "scf.norms", 2 * sizeof(double), &pn));
  double *q = static_cast<double*>(pq), *qo = static_cast<double*>(pqo), *r = static_cast<double*>(pr);
  double* u = static_cast<double*>(pu);
  double* norms = static_cast<double*>(pn);
  const int m = anderson ? so->history : 0;
  double *Qh = nullptr, *Rh = nullptr, *G = nullptr, *cf = nullptr, *Ph = nullptr;
  if (so->mixer == SP2_MIX_ANDERSON_MLP) {
    void* a;
    TRY(ws(h, "scf.Ph", (size_t)m * tot * sizeof(double), &a));
    Ph = static_cast<double*>(a);
  }
  if (m > 0) {
    void *a, *b, *c2, *d;
    TRY(ws(h, "scf.Qh", (size_t)m * tot * sizeof(double), &a));
    TRY(ws(h, "scf.Rh", (size_t)m * tot * sizeof(double), &b));
    TRY(ws(h, "scf.G", (size_t)F * m * m * sizeof(double), &c2));
    TRY(ws(h, "scf.c", (size_t)F * m * sizeof(double), &d));
    Qh = static_cast<double*>(a);
    Rh = static_cast<double*>(b);
    G = static_cast<double*>(c2);
    cf = static_cast<double*>(d);
  }
  float *mx = nullptr, *my = nullptr, *mh = nullptr;
  double* nr = nullptr;
  if (learned) {
    void *a, *b, *c2, *d;
    TRY(ws(h, "scf.mx", tot * sizeof(float), &a));
    TRY(ws(h, "scf.my", tot * sizeof(float), &b));
    TRY(ws(h, "scf.mh", (size_t)F * so->hidden * sizeof(float), &c2));
    TRY(ws(h, "scf.nr", F * sizeof(double), &d));
    mx = static_cast<float*>(a);
    my = static_cast<float*>(b);
    mh = static_cast<float*>(c2);
    nr = static_cast<double*>(d);
  }
  CK(cudaMemsetAsync(q, 0, tot * sizeof(double), h->stream));
  Ctx c;
  TRY(make_ctx(h, o.mode, N, np, o.time_kernels != 0, &c));
  MatBuf X[2], Y[2];
  double norm0 = 0.0;
  int it = 0;
  bool done = false;
  std::vector<double> Gh, ch;
  FermiState fs;               // finite T: the recursion's history, set up once per arithmetic
  if (finite_t) TRY(fermi_setup(c, fs, Hd, N, dtype, so->mu, so->kT, ndbl, so->canonical != 0, true));
  std::vector<int8_t> frozen;  // branch signs of the SP2 run that fixed the polynomial
  bool frozen_here = false;    // the fixed polynomial is this loop's (not the caller's)
  int a0 = 0;                  // first iteration of the current Anderson history
  int refine_iter = -1;        // first iteration computed in refine_mode
  double best = 0.0;           // smallest residual so far and iterations since it
  int since_best = 0;
  for (; it < so->max_iter && !done; ++it) {
    // u = V + K q, perturbation diag(u (x) 1_norb), response, site charges
    CK(launch_site_potential(static_cast<const double*>(Vd), static_cast<const double*>(Kd), q, F,
                             ns, u, h->stream));
    CK(launch_expand_sites(u, F, ns, norb, pub, dtype, h->stream));
    c.kernels += 2;
    if (finite_t) {
      // one finite-temperature response per field through the kept history
      const size_t per = (size_t)N * dsize(dtype);
      for (int64_t f = 0; f < F; ++f) {
        FMat* r;
        TRY(fermi_response(c, fs, static_cast<const char*>(pub) + f * per, dtype, 1, false, &r));
        CK(launch_site_charges(r->m.master, o.mode, 1, ns, norb, np, qo + f * ns, h->stream));
        c.kernels++;
      }
    } else {
    Sp2Out rr;
    TRY(run_sp2(h, Hd, N, dtype, nocc, o, pub, F, 1, false, X, Y, c, &rr));
    if (!rr.converged) return fail(h, SP2_ENOCONV, "SP2 did not converge inside the SCF loop");
    TRY(poll_state(h));   // the branch signs of this run (read below)
    if (o.fixed_m == 0) {
      // H is the same in every iteration: later iterations apply this run's polynomial
      // -- its branches, M and spectral bounds -- so the response map changes only by
      // rounding from one iteration to the next
      frozen_here = true;
      frozen.resize(rr.M);
      for (int i = 1; i <= rr.M; ++i) frozen[i - 1] = (int8_t)h->h_state->sigma[i];
      o.fixed_m = rr.M;
      o.sigma_in = frozen.data();
      o.eps_min = rr.emin;
      o.eps_max = rr.emax;
    }
    CK(launch_site_charges(rr.yout.master, o.mode, F, ns, norb, np, qo, h->stream));
    }
    CK(cudaMemsetAsync(norms, 0, 2 * sizeof(double), h->stream));
    CK(launch_residual(qo, q, tot, r, norms, h->stream));
    c.kernels += 2;
    if (traj_r) CK(cudaMemcpyAsync(traj_r + (size_t)it * tot, r, tot * sizeof(double),
                                   cudaMemcpyDeviceToDevice, h->stream));
    if (traj_q) CK(cudaMemcpyAsync(traj_q + (size_t)it * tot, q, tot * sizeof(double),
                                   cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(h->h_state->bounds, norms, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const double s1 = h->h_state->bounds[0], s2 = h->h_state->bounds[1];
    if (it == 0) norm0 = std::sqrt(s2);
    const double res = norm0 > 0.0 ? std::sqrt(s1) / norm0 : std::sqrt(s1);
    if (residuals) residuals[it] = res;
    if (!std::isfinite(res)) return fail(h, SP2_ENONFINITE, "non-finite SCF residual");
    if (res <= so->tol) {
      done = true;
      break;
    }
    if (it == 0 || res < best) {
      best = res;
      since_best = 0;
    } else {
      ++since_best;
    }
    if (refine && refine_iter < 0 && (res <= so->refine_below || since_best >= 3)) {
      // the following iterations compute the responses in refine_mode
      o.mode = so->refine_mode;
      TRY(make_ctx(h, o.mode, N, np, o.time_kernels != 0, &c));
      if (frozen_here && so->refine_mode == SP2_MODE_FP64) {
        // FP64 converges its own SP2 polynomial once (stop rule, to its tighter floor),
        // which is then fixed again. Other arithmetic keeps the polynomial of the split
        // run: a precision floor reached earlier would shorten it and move the response
        // map (the residual jumps to the difference of the two maps).
        o.fixed_m = 0;
        o.sigma_in = nullptr;
        o.eps_min = o.eps_max = 0.0;
      }
      if (finite_t)
        TRY(fermi_setup(c, fs, Hd, N, dtype, so->mu, so->kT, ndbl, so->canonical != 0, true));
      refine_iter = it + 1;
      a0 = it + 1;  // the new Anderson history holds only residuals of the refined arithmetic
      since_best = 0;
    }
    if (so->mixer == SP2_MIX_LINEAR || (anderson && it < a0)) {
      CK(launch_axpy_d(q, so->alpha, r, tot, h->stream));
      c.kernels++;
    } else if (anderson) {
      const int ia = it - a0;
      const int slot = ia % m, me = ia + 1 < m ? ia + 1 : m;
      CK(cudaMemcpyAsync(Qh + (size_t)slot * tot, q, tot * sizeof(double), cudaMemcpyDeviceToDevice,
                         h->stream));
      CK(cudaMemcpyAsync(Rh + (size_t)slot * tot, r, tot * sizeof(double), cudaMemcpyDeviceToDevice,
                         h->stream));
      if (Ph) {
        // the learned step as Anderson's preconditioner: P(r) = alpha r + ||r|| MLP(r / ||r||)
        double* p = Ph + (size_t)slot * tot;
        CK(launch_normalise_rows(r, F, ns, mx, nr, h->stream));
        TRY(mlp_fwd(h, so->W1, so->W2, (int)ns, so->hidden, mx, F, mh, my, so->bf16_infer));
        CK(cudaMemsetAsync(p, 0, tot * sizeof(double), h->stream));
        CK(launch_axpy_d(p, so->alpha, r, tot, h->stream));
        CK(launch_apply_update(p, my, nr, F, ns, h->stream));
        c.kernels += 5;
      }
      CK(launch_gram(Rh, me, F, ns, tot, G, h->stream));
      Gh.resize((size_t)F * me * me);
      ch.resize((size_t)F * me);
      CK(cudaMemcpyAsync(Gh.data(), G, Gh.size() * sizeof(double), cudaMemcpyDeviceToHost,
                         h->stream));
      CK(cudaStreamSynchronize(h->stream));
      for (int64_t f = 0; f < F; ++f) anderson_coeffs(&Gh[(size_t)f * me * me], me, &ch[(size_t)f * me]);
      CK(cudaMemcpyAsync(cf, ch.data(), ch.size() * sizeof(double), cudaMemcpyHostToDevice,
                         h->stream));
      // q = sum_i c_i (q_i + alpha r_i), or sum_i c_i (q_i + P(r_i)) with the learned step
      CK(launch_anderson_combine(Qh, Ph ? Ph : Rh, cf, me, F, ns, tot, Ph ? 1.0 : so->alpha, q,
                                 h->stream));
      CK(cudaStreamSynchronize(h->stream));  // ch is reused next iteration
      c.kernels += 2;
    } else {
      // q <- q + alpha r + ||r|| MLP(r / ||r||): a learned correction to linear mixing
      CK(launch_normalise_rows(r, F, ns, mx, nr, h->stream));
      TRY(mlp_fwd(h, so->W1, so->W2, (int)ns, so->hidden, mx, F, mh, my, so->bf16_infer));
      CK(launch_axpy_d(q, so->alpha, r, tot, h->stream));
      CK(launch_apply_update(q, my, nr, F, ns, h->stream));
      c.kernels += 5;
    }
  }
  if (iterations) *iterations = done ? it + 1 : it;
  CK(cudaMemcpyAsync(oq.dev, q, tot * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  TRY(finish_out(h, oq));
  CK(cudaStreamSynchronize(h->stream));
  if (info) {
    info->converged = done ? 1 : 0;
    info->M = 0;
    info->refine_iter = refine_iter;
  }
  fill_timing(c, 1 << 30, info);
  if (!done) return fail(h, SP2_ENOCONV, "SCF residual above tol after %d iterations", so->max_iter);
  return SP2_OK;
}

}  // extern "C"
