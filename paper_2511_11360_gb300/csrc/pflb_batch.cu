// C ABI of the batched step (declared in include/pflb.h): many 2D domains
// advanced by one persistent launch per time level, optional CUDA-graph
// replay, and an autotuner of the launch shape.
#include <algorithm>
#include <cinttypes>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pflb_internal.h"

using namespace pflb;

constexpr int kBatchFams = 5;   // the fused-step families 0..4

struct pflb_batch {
  std::vector<pflb_handle*> dom;
  cudaStream_t stream = nullptr;   // the caller's stream (every domain's)
  cudaStream_t gstream = nullptr;  // internal stream the graphs replay on
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  pflb_batch_launch cfg = {128, 16, 0, 0, 0.0};
  int grid = 0;                    // resident blocks the launch shape allows (every family's kernel)
  int fam_t0[kBatchFams] = {};      // the families' ranges of the tile list
  int fam_n[kBatchFams] = {};
  int fgrid[kBatchFams] = {};       // persistent blocks of each family's kernel
  cudaStream_t fstream[kBatchFams] = {};   // branches of a step (the first family runs on the step's stream)
  cudaEvent_t ev_fork = nullptr, ev_gamma = nullptr, ev_join[kBatchFams] = {};
  int ggrid = 0;                   // blocks of the gamma pre-pass
  BatchTile* d_tiles = nullptr;
  int ntiles = 0;
  BatchGammaEntry* d_gent = nullptr;
  int ngent = 0;
  StepArgs* d_args = nullptr;      // 2 x n: arguments of the next step and the one after
  unsigned* d_counter = nullptr;   // tile claim counters of those two steps, one per family
  DevObs** d_obs_src = nullptr;
  DevObs* d_obs_out = nullptr;
  bool layout_ok = false, tables_ok = false;
  std::vector<long long> exp_step;
  std::vector<int> exp_cur;
  int ph = 0;                      // which of the two argument tables the next step uses
  bool use_graph = false;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  long long cells = 0;
  int status = PFLB_OK;
  char err[512] = {0};
};

namespace {

constexpr int kGammaEntryCells = 8192;

int bfail(pflb_batch* b, int code, const char* fmt, ...) {
  if (b) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->err, sizeof(b->err), fmt, ap);
    va_end(ap);
    if (b->status == PFLB_OK || code == PFLB_EUNSTABLE) b->status = code;
  }
  return code;
}

#define BCU(b, call)                                                                   \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return bfail((b), PFLB_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

int n_of(const pflb_batch* b) { return (int)b->dom.size(); }

void drop_graphs(pflb_batch* b) {
  for (auto& g : b->gexec) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

template <typename T>
int upload(pflb_batch* b, T** dst, const std::vector<T>& src) {
  cudaFree(*dst);
  *dst = nullptr;
  if (src.empty()) return PFLB_OK;
  if (cudaMalloc(dst, src.size() * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, PFLB_ENOMEM, "cudaMalloc of %zu bytes failed", src.size() * sizeof(T));
  }
  BCU(b, cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return PFLB_OK;
}

// Work lists for the current launch shape: the tiles of the step kernel and
// the cell ranges of the gamma pre-pass.
int build_layout(pflb_batch* b) {
  // The old lists may still be read by launches in flight.
  BCU(b, cudaStreamSynchronize(b->stream));
  BCU(b, cudaStreamSynchronize(b->gstream));
  const int ta = b->cfg.tile_a, ch = b->cfg.chunk;
  std::vector<BatchTile> tiles;
  std::vector<BatchGammaEntry> gent;
  for (int i = 0; i < n_of(b); ++i) {
    const pflb_handle* h = b->dom[i];
    const int nx = h->prm.nx, ny = h->prm.ny;
    for (int c0 = 0; c0 < ny; c0 += ch)
      for (int a0 = 0; a0 < nx; a0 += ta) tiles.push_back(BatchTile{i, a0, c0, h->family});
    if (handle_nonlocal(h))
      for (long long s = 0; s < h->N; s += kGammaEntryCells)
        gent.push_back(BatchGammaEntry{i, (int)s, (int)(s + kGammaEntryCells < h->N ? s + kGammaEntryCells : h->N), 0});
  }
  // Tiles of one family together: resident blocks then run the same branch
  // of the kernel's family dispatch (one family's code in the instruction
  // cache at a time). The order of tiles within a step does not change the
  // state.
  std::stable_sort(tiles.begin(), tiles.end(),
                   [](const BatchTile& x, const BatchTile& y) { return x.fam < y.fam; });
  int rc = upload(b, &b->d_tiles, tiles);
  if (rc) return rc;
  if ((rc = upload(b, &b->d_gent, gent))) return rc;
  b->ntiles = (int)tiles.size();
  b->ngent = (int)gent.size();
  for (int f = 0; f < kBatchFams; ++f) b->fam_t0[f] = b->fam_n[f] = 0;
  for (int t = 0; t < b->ntiles; ++t) {
    const int f = tiles[t].fam;
    if (b->fam_n[f]++ == 0) b->fam_t0[f] = t;
  }
  const int sms = num_sms();
  b->grid = 0;
  for (int f = 0; f < kBatchFams; ++f) {
    const int maxb = batch_max_blocks_per_sm(ta, f);
    int bps = b->cfg.blocks_per_sm > 0 ? b->cfg.blocks_per_sm : maxb;
    if (bps > maxb) bps = maxb;
    long long grid = (long long)bps * sms;
    if (grid > b->fam_n[f]) grid = b->fam_n[f];
    b->fgrid[f] = (int)grid;
    if (b->fgrid[f] > b->grid) b->grid = b->fgrid[f];
  }
  b->ggrid = b->ngent < 4 * sms ? (b->ngent > 0 ? b->ngent : 1) : 4 * sms;
  drop_graphs(b);
  b->layout_ok = true;
  return PFLB_OK;
}

// Arguments of domain h for the step k time levels ahead (k = 0 or 1). The
// state alternates between two buffers and every per-step slot (AA parity,
// observables ring of 2, gamma pair) has period 2, so two tables serve every
// step once built.
StepArgs args_ahead(const pflb_handle* h, int k, int chunk) {
  StepArgs a = handle_step_args(h);
  const long long s = h->step + k;
  const int cur = h->cur ^ (k & 1);
  a.g_src = h->g[cur];
  a.g_dst = h->g[1 - cur];
  a.parity = (int)(s & 1);
  a.chunk = chunk;
  a.obs_slot = h->obs + (s % h->obs_cap);
  a.obs_zero = h->obs + ((s + 1) % h->obs_cap);
  if (handle_nonlocal(h)) {
    a.gamma_acc = h->gamma_acc + 2 * (s & 1);
    a.gamma_next = h->gamma_acc + 2 * ((s + 1) & 1);
  }
  return a;
}

int build_tables(pflb_batch* b) {
  const int n = n_of(b);
  std::vector<StepArgs> t(2 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    t[i] = args_ahead(b->dom[i], 0, b->cfg.chunk);
    t[n + i] = args_ahead(b->dom[i], 1, b->cfg.chunk);
    b->exp_step[i] = b->dom[i]->step;
    b->exp_cur[i] = b->dom[i]->cur;
  }
  BCU(b, cudaMemcpyAsync(b->d_args, t.data(), t.size() * sizeof(StepArgs), cudaMemcpyHostToDevice, b->stream));
  BCU(b, cudaMemsetAsync(b->d_counter, 0, 2 * kBatchFams * sizeof(unsigned), b->stream));
  BCU(b, cudaStreamSynchronize(b->stream));
  b->ph = 0;
  b->tables_ok = true;
  return PFLB_OK;
}

int prepare(pflb_batch* b) {
  for (int i = 0; i < n_of(b); ++i) {
    const pflb_handle* h = b->dom[i];
    if (!h->initialized) return bfail(b, PFLB_EINVAL, "domain %d is not initialised", i);
    if (h->status != PFLB_OK && h->status != PFLB_EUNSTABLE)
      return bfail(b, h->status, "domain %d: %s", i, h->err);
  }
  int rc;
  if (!b->layout_ok && (rc = build_layout(b))) return rc;
  bool fresh = b->tables_ok;
  for (int i = 0; fresh && i < n_of(b); ++i)
    fresh = b->dom[i]->step == b->exp_step[i] && b->dom[i]->cur == b->exp_cur[i];
  if (!fresh && (rc = build_tables(b))) return rc;
  return PFLB_OK;
}

// One batched step using argument table k, on stream s: the gamma pre-pass,
// then one kernel per family present, forked on the family streams after the
// pre-pass and joined back into s (the same dependencies in a captured graph).
// The nonlocal family whose kernel runs on the step's own stream (the first
// of Chai2018, Hu2019 present), or -1.
int first_nonlocal(const pflb_batch* b) {
  if (b->fam_n[FAM_CHAI] > 0) return FAM_CHAI;
  if (b->fam_n[FAM_HU] > 0) return FAM_HU;
  return -1;
}

void launch_one(pflb_batch* b, int k, cudaStream_t s) {
  const int n = n_of(b);
  // One step as a fork / join over the families' kernels. Every branch
  // starts after the previous step (the fork on s); the nonlocal families
  // (Chai2018, Hu2019) also wait for the gamma pre-pass on s, while the
  // local ones run beside it on their own streams.
  cudaEventRecord(b->ev_fork, s);
  auto args_of = [&](int f) {
    BatchArgs ba;
    ba.args = b->d_args + (size_t)k * n;
    ba.tiles = b->d_tiles + b->fam_t0[f];
    ba.ntiles = b->fam_n[f];
    ba.ninst = n;
    ba.chunk = b->cfg.chunk;
    ba.counter = b->d_counter + k * kBatchFams + f;
    ba.counter_next = b->d_counter + (1 - k) * kBatchFams + f;
    return ba;
  };
  auto branch = [&](int f, cudaEvent_t after) {
    cudaStream_t sf = b->fstream[f];
    cudaStreamWaitEvent(sf, after, 0);
    batch_step(b->cfg.tile_a, f, args_of(f), b->fgrid[f], sf);
    cudaEventRecord(b->ev_join[f], sf);
  };
  for (int f = 0; f < kBatchFams; ++f)
    if (b->fam_n[f] > 0 && f != FAM_CHAI && f != FAM_HU) branch(f, b->ev_fork);
  if (b->ngent > 0) {
    BatchGammaArgs ga;
    ga.args = b->d_args + (size_t)k * n;
    ga.ent = b->d_gent;
    ga.nent = b->ngent;
    ga.ninst = n;
    batch_gamma(ga, b->ggrid, s);
  }
  cudaEventRecord(b->ev_gamma, s);
  bool on_s = false;   // the first nonlocal family runs on s itself
  for (int f : {FAM_CHAI, FAM_HU}) {
    if (b->fam_n[f] == 0) continue;
    if (!on_s) {
      batch_step(b->cfg.tile_a, f, args_of(f), b->fgrid[f], s);
      on_s = true;
    } else {
      branch(f, b->ev_gamma);
    }
  }
  for (int f = 0; f < kBatchFams; ++f) {
    const bool side = b->fam_n[f] > 0 && !((f == FAM_CHAI || f == FAM_HU) && f == first_nonlocal(b));
    if (side) cudaStreamWaitEvent(s, b->ev_join[f], 0);
  }
}

int capture_graphs(pflb_batch* b) {
  for (int k0 = 0; k0 < 2; ++k0) {
    if (b->gexec[k0]) continue;
    cudaGraph_t g = nullptr;
    BCU(b, cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal));
    launch_one(b, k0, b->gstream);
    launch_one(b, 1 - k0, b->gstream);
    BCU(b, cudaStreamEndCapture(b->gstream, &g));
    cudaError_t e = cudaGraphInstantiate(&b->gexec[k0], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->gexec[k0] = nullptr;
      return bfail(b, PFLB_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
    }
  }
  return PFLB_OK;
}

// Advance every domain n steps (graphs as configured).
int step_impl(pflb_batch* b, long long n, bool graphs) {
  int rc = prepare(b);
  if (rc) return rc;
  if (n <= 0) return PFLB_OK;
  long long done = 0;
  if (graphs && n >= 2) {
    if ((rc = capture_graphs(b))) return rc;
    BCU(b, cudaEventRecord(b->ev_in, b->stream));
    BCU(b, cudaStreamWaitEvent(b->gstream, b->ev_in, 0));
    for (; n - done >= 2; done += 2) BCU(b, cudaGraphLaunch(b->gexec[b->ph], b->gstream));
    if (done < n) {
      launch_one(b, b->ph, b->gstream);
      b->ph ^= 1;
      ++done;
    }
    BCU(b, cudaEventRecord(b->ev_out, b->gstream));
    BCU(b, cudaStreamWaitEvent(b->stream, b->ev_out, 0));
  } else {
    for (; done < n; ++done) {
      launch_one(b, b->ph, b->stream);
      b->ph ^= 1;
    }
  }
  BCU(b, cudaGetLastError());
  for (int i = 0; i < n_of(b); ++i) {
    pflb_handle* h = b->dom[i];
    h->step += n;
    h->cur ^= (int)(n & 1);
    b->exp_step[i] = h->step;
    b->exp_cur[i] = h->cur;
  }
  return PFLB_OK;
}

int gather_obs(pflb_batch* b, std::vector<pflb_obs>& out) {
  const int n = n_of(b);
  std::vector<DevObs*> src(n);
  for (int i = 0; i < n; ++i) {
    const pflb_handle* h = b->dom[i];
    const long long s = h->step > 0 ? h->step - 1 : 0;
    src[i] = h->obs + (s % h->obs_cap);
  }
  BCU(b, cudaMemcpyAsync(b->d_obs_src, src.data(), n * sizeof(DevObs*), cudaMemcpyHostToDevice, b->stream));
  batch_obs_gather(b->d_obs_src, b->d_obs_out, n, b->stream);
  BCU(b, cudaGetLastError());
  std::vector<DevObs> d(n);
  BCU(b, cudaMemcpyAsync(d.data(), b->d_obs_out, n * sizeof(DevObs), cudaMemcpyDeviceToHost, b->stream));
  BCU(b, cudaStreamSynchronize(b->stream));
  out.resize(n);
  int rc = PFLB_OK;
  for (int i = 0; i < n; ++i) {
    const pflb_handle* h = b->dom[i];
    obs_to_host(d[i], h->step > 0 ? h->step - 1 : 0, &out[i]);
    if (out[i].status != PFLB_OK && rc == PFLB_OK)
      rc = bfail(b, PFLB_EUNSTABLE, "domain %d: step %" PRId64 " produced rho <= 0 or non-finite phi/u", i,
                 out[i].step);
  }
  return rc;
}

// ---- autotuner --------------------------------------------------------------

std::string signature(const pflb_batch* b) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  memset(&prop, 0, sizeof(prop));
  cudaGetDeviceProperties(&prop, dev);
  uint64_t hsh = 1469598103934665603ull;  // FNV-1a over (nx, ny, family, bc_y)
  auto mix = [&](int v) {
    for (int k = 0; k < 4; ++k) {
      hsh ^= (uint64_t)((v >> (8 * k)) & 0xff);
      hsh *= 1099511628211ull;
    }
  };
  for (const pflb_handle* h : b->dom) {
    mix(h->prm.nx);
    mix(h->prm.ny);
    mix(h->family);
    mix(h->prm.bc_y);
  }
  std::string name(prop.name);
  for (auto& c : name)
    if (c == ' ') c = '_';
  char buf[256];
  snprintf(buf, sizeof(buf), "%s/sm%d/n%d/%016" PRIx64, name.c_str(), prop.multiProcessorCount, n_of(b), hsh);
  return buf;
}

bool cache_lookup(const char* path, const std::string& sig, pflb_batch_launch* cfg) {
  if (!path) return false;
  FILE* fp = fopen(path, "r");
  if (!fp) return false;
  char line[512], key[320];
  bool found = false;
  while (fgets(line, sizeof(line), fp)) {
    pflb_batch_launch c = {0, 0, 0, 1, 0.0};
    if (sscanf(line, "%319s %d %d %d %lf", key, &c.tile_a, &c.chunk, &c.blocks_per_sm, &c.ms_per_step) == 5 &&
        sig == key && batch_tile_supported(c.tile_a) && c.chunk >= 1 && c.blocks_per_sm >= 0) {
      *cfg = c;
      found = true;  // the last matching line wins
    }
  }
  fclose(fp);
  return found;
}

void cache_store(const char* path, const std::string& sig, const pflb_batch_launch& c) {
  if (!path) return;
  FILE* fp = fopen(path, "a");
  if (!fp) return;
  fprintf(fp, "%s %d %d %d %.6f\n", sig.c_str(), c.tile_a, c.chunk, c.blocks_per_sm, c.ms_per_step);
  fclose(fp);
}

// Raw copy of every domain's state (source g, f, phi*u, observables ring,
// gamma pairs) into one device buffer, and back.
struct Snapshot {
  char* buf = nullptr;
  std::vector<long long> step;
  std::vector<int> cur;
};

template <typename F>
void for_each_piece(pflb_batch* b, F fn) {
  size_t off = 0;
  for (pflb_handle* h : b->dom) {
    // Population arrays hold Q x (N rounded up to the layout block).
    const size_t npad = (size_t)((h->N + kPopBlock - 1) / kPopBlock) * kPopBlock;
    const size_t ng = (size_t)h->QG * npad * h->elem, nf = (size_t)h->QF * npad * h->elem;
    fn(h, 0, off, ng);
    off += ng;
    fn(h, 1, off, nf);
    off += nf;
    if (h->phiu) {
      const size_t np = (size_t)h->dim * h->N * sizeof(float);
      fn(h, 2, off, np);
      off += np;
    }
    const size_t no = (size_t)(h->obs_cap + 1) * sizeof(DevObs);
    fn(h, 3, off, no);
    off += no;
    fn(h, 4, off, 6 * sizeof(double));
    off += 6 * sizeof(double);
  }
  fn(nullptr, -1, off, 0);
}

void* piece_ptr(pflb_handle* h, int which, int cur) {
  switch (which) {
    case 0: return h->g[cur];
    case 1: return h->f;
    case 2: return h->phiu;
    case 3: return h->obs;
    default: return h->gamma_acc;
  }
}

int snapshot_take(pflb_batch* b, Snapshot& s) {
  size_t total = 0;
  for_each_piece(b, [&](pflb_handle* h, int, size_t off, size_t) {
    if (!h) total = off;
  });
  if (cudaMalloc(&s.buf, total) != cudaSuccess) {
    cudaGetLastError();
    s.buf = nullptr;
    return bfail(b, PFLB_ENOMEM, "autotune: cudaMalloc of %zu bytes for the state snapshot failed", total);
  }
  cudaError_t err = cudaSuccess;
  for_each_piece(b, [&](pflb_handle* h, int which, size_t off, size_t bytes) {
    if (!h || err != cudaSuccess) return;
    err = cudaMemcpyAsync(s.buf + off, piece_ptr(h, which, h->cur), bytes, cudaMemcpyDeviceToDevice, b->stream);
  });
  BCU(b, err);
  for (pflb_handle* h : b->dom) {
    s.step.push_back(h->step);
    s.cur.push_back(h->cur);
  }
  return PFLB_OK;
}

int snapshot_restore(pflb_batch* b, Snapshot& s) {
  cudaError_t err = cudaSuccess;
  int i = 0;
  for (pflb_handle* h : b->dom) {
    h->step = s.step[i];
    h->cur = s.cur[i];
    ++i;
  }
  for_each_piece(b, [&](pflb_handle* h, int which, size_t off, size_t bytes) {
    if (!h || err != cudaSuccess) return;
    err = cudaMemcpyAsync(piece_ptr(h, which, h->cur), s.buf + off, bytes, cudaMemcpyDeviceToDevice, b->stream);
  });
  cudaError_t e2 = cudaStreamSynchronize(b->stream);
  cudaFree(s.buf);
  s.buf = nullptr;
  BCU(b, err);
  BCU(b, e2);
  b->tables_ok = false;
  return PFLB_OK;
}

int set_cfg(pflb_batch* b, const pflb_batch_launch& c) {
  if (!batch_tile_supported(c.tile_a)) return bfail(b, PFLB_EINVAL, "tile_a must be 64, 128 or 256");
  if (c.chunk < 1) return bfail(b, PFLB_EINVAL, "chunk must be >= 1");
  if (c.blocks_per_sm < 0) return bfail(b, PFLB_EINVAL, "blocks_per_sm must be >= 0");
  if (c.tile_a != b->cfg.tile_a || c.chunk != b->cfg.chunk || c.blocks_per_sm != b->cfg.blocks_per_sm)
    b->layout_ok = false;
  b->cfg.tile_a = c.tile_a;
  b->cfg.chunk = c.chunk;
  b->cfg.blocks_per_sm = c.blocks_per_sm;
  b->cfg.from_cache = c.from_cache;
  b->cfg.ms_per_step = c.ms_per_step;
  return PFLB_OK;
}

}  // namespace

extern "C" {

int pflb_batch_create(const pflb_params* params, int32_t n, void* cuda_stream, pflb_batch** out) {
  if (!out) return PFLB_EINVAL;
  *out = nullptr;
  pflb_batch* b = new (std::nothrow) pflb_batch();
  if (!b) return PFLB_ENOMEM;
  *out = b;
  if (!params || n < 1) return bfail(b, PFLB_EINVAL, "need params and n >= 1");
  for (int i = 0; i < n; ++i) {
    if (params[i].dim != 2) return bfail(b, PFLB_EINVAL, "domain %d: the batched step is 2D only", i);
    if (params[i].storage != PFLB_FP32) return bfail(b, PFLB_EINVAL, "domain %d: the batched step needs FP32 storage", i);
    if (params[i].family > PFLB_CAC_LIANG2018)
      return bfail(b, PFLB_EINVAL, "domain %d: the batched step runs the fused-kernel families (0..4)", i);
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return bfail(b, PFLB_ECUDA, "no CUDA device");
  }
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->dom.reserve(n);
  for (int i = 0; i < n; ++i) {
    pflb_params p = params[i];
    p.obs_capacity = 2;
    pflb_handle* h = nullptr;
    int rc = pflb_create(&p, cuda_stream, &h);
    if (rc != PFLB_OK) {
      bfail(b, rc, "domain %d: %s", i, h ? h->err : "create failed");
      pflb_destroy(h);
      return rc;
    }
    b->dom.push_back(h);
    b->cells += h->N;
  }
  b->exp_step.assign(n, -1);
  b->exp_cur.assign(n, 0);
  BCU(b, cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking));
  BCU(b, cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
  BCU(b, cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
  BCU(b, cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
  BCU(b, cudaEventCreateWithFlags(&b->ev_gamma, cudaEventDisableTiming));
  for (int f = 0; f < kBatchFams; ++f) {
    BCU(b, cudaStreamCreateWithFlags(&b->fstream[f], cudaStreamNonBlocking));
    BCU(b, cudaEventCreateWithFlags(&b->ev_join[f], cudaEventDisableTiming));
  }
  auto alloc = [&](void** p, size_t bytes) -> int {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, PFLB_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
    }
    return PFLB_OK;
  };
  int rc;
  if ((rc = alloc((void**)&b->d_args, 2 * (size_t)n * sizeof(StepArgs)))) return rc;
  if ((rc = alloc((void**)&b->d_counter, 2 * kBatchFams * sizeof(unsigned)))) return rc;
  if ((rc = alloc((void**)&b->d_obs_src, (size_t)n * sizeof(DevObs*)))) return rc;
  if ((rc = alloc((void**)&b->d_obs_out, (size_t)n * sizeof(DevObs)))) return rc;
  BCU(b, cudaMemset(b->d_counter, 0, 2 * kBatchFams * sizeof(unsigned)));
  return PFLB_OK;
}

int32_t pflb_batch_size(const pflb_batch* b) { return b ? (int32_t)b->dom.size() : 0; }

pflb_handle* pflb_batch_domain(pflb_batch* b, int32_t i) {
  if (!b || i < 0 || i >= n_of(b)) return nullptr;
  return b->dom[i];
}

int pflb_batch_init(pflb_batch* b, int32_t i, const float* phi0, const float* u0) {
  if (!b) return PFLB_EINVAL;
  if (i < 0 || i >= n_of(b)) return bfail(b, PFLB_EINVAL, "domain index %d out of range", i);
  const int rc = pflb_init(b->dom[i], phi0, u0);
  if (rc != PFLB_OK) return bfail(b, rc, "domain %d: %s", i, b->dom[i]->err);
  return PFLB_OK;
}

int pflb_batch_step(pflb_batch* b, int64_t nsteps) {
  if (!b) return PFLB_EINVAL;
  if (nsteps < 0) return bfail(b, PFLB_EINVAL, "nsteps must be >= 0");
  if (b->status != PFLB_OK && b->status != PFLB_EUNSTABLE) return b->status;
  const NvtxRange range("pflb_batch_step");
  return step_impl(b, nsteps, b->use_graph);
}

int pflb_batch_set_graph(pflb_batch* b, int32_t on) {
  if (!b) return PFLB_EINVAL;
  b->use_graph = on != 0;
  return PFLB_OK;
}

int pflb_batch_set_launch(pflb_batch* b, const pflb_batch_launch* cfg) {
  if (!b || !cfg) return b ? bfail(b, PFLB_EINVAL, "null argument") : PFLB_EINVAL;
  pflb_batch_launch c = *cfg;
  c.from_cache = 0;
  c.ms_per_step = 0.0;
  return set_cfg(b, c);
}

int pflb_batch_get_launch(const pflb_batch* b, pflb_batch_launch* out) {
  if (!b || !out) return PFLB_EINVAL;
  *out = b->cfg;
  return PFLB_OK;
}

int pflb_batch_autotune(pflb_batch* b, int32_t steps_per_trial, const char* cache_path, pflb_batch_launch* out) {
  if (!b) return PFLB_EINVAL;
  if (steps_per_trial < 1) return bfail(b, PFLB_EINVAL, "steps_per_trial must be >= 1");
  if (b->status != PFLB_OK && b->status != PFLB_EUNSTABLE) return b->status;
  const std::string sig = signature(b);
  pflb_batch_launch best = {0, 0, 0, 0, 0.0};
  int rc;
  if (cache_lookup(cache_path, sig, &best)) {
    if ((rc = set_cfg(b, best))) return rc;
    if (out) *out = b->cfg;
    return PFLB_OK;
  }
  if ((rc = prepare(b))) return rc;
  Snapshot snap;
  if ((rc = snapshot_take(b, snap))) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const pflb_batch_launch keep = b->cfg;
  double best_ms = -1.0;
  static const int tas[3] = {64, 128, 256};
  static const int chunks[4] = {8, 16, 32, 64};
  for (int ta : tas) {
    int maxb = 1;
    for (int f = 0; f < kBatchFams; ++f)
      maxb = batch_max_blocks_per_sm(ta, f) > maxb ? batch_max_blocks_per_sm(ta, f) : maxb;
    const int bpss[2] = {0, maxb / 2};
    for (int ci = 0; ci < 4 && rc == PFLB_OK; ++ci) {
      for (int bi = 0; bi < 2 && rc == PFLB_OK; ++bi) {
        if (bi == 1 && (bpss[1] < 1 || bpss[1] == maxb)) continue;
        pflb_batch_launch c = {ta, chunks[ci], bpss[bi], 0, 0.0};
        if ((rc = set_cfg(b, c))) break;
        if ((rc = step_impl(b, 1, false))) break;  // warm-up (and layout upload)
        cudaEventRecord(e0, b->stream);
        if ((rc = step_impl(b, steps_per_trial, false))) break;
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          cudaGetLastError();
          rc = bfail(b, PFLB_ECUDA, "autotune: timing failed");
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = (double)ms / steps_per_trial;
        if (best_ms < 0.0 || per < best_ms) {
          best_ms = per;
          best = c;
          best.ms_per_step = per;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int rr = snapshot_restore(b, snap);
  if (rc == PFLB_OK) rc = rr;
  if (rc != PFLB_OK) {
    set_cfg(b, keep);
    return rc;
  }
  if ((rc = set_cfg(b, best))) return rc;
  cache_store(cache_path, sig, best);
  if (out) *out = b->cfg;
  return PFLB_OK;
}

int pflb_batch_observables(pflb_batch* b, pflb_obs* out) {
  if (!b || !out) return b ? bfail(b, PFLB_EINVAL, "null argument") : PFLB_EINVAL;
  std::vector<pflb_obs> o;
  const int rc = gather_obs(b, o);
  if (!o.empty()) memcpy(out, o.data(), o.size() * sizeof(pflb_obs));
  return rc;
}

int pflb_batch_sync(pflb_batch* b) {
  if (!b) return PFLB_EINVAL;
  std::vector<pflb_obs> o;
  return gather_obs(b, o);
}

int64_t pflb_batch_cells(const pflb_batch* b) { return b ? b->cells : -1; }

double pflb_batch_bytes_per_step(const pflb_batch* b) {
  if (!b) return 0.0;
  double s = 0.0;
  for (const pflb_handle* h : b->dom) s += pflb_bytes_per_update(h) * (double)h->N;
  return s;
}

int pflb_batch_destroy(pflb_batch* b) {
  if (!b) return PFLB_OK;
  if (b->stream || b->gstream) {
    cudaStreamSynchronize(b->stream);
    if (b->gstream) cudaStreamSynchronize(b->gstream);
  }
  drop_graphs(b);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  for (int f = 0; f < kBatchFams; ++f) {
    if (b->fstream[f]) {
      cudaStreamSynchronize(b->fstream[f]);
      cudaStreamDestroy(b->fstream[f]);
    }
    if (b->ev_join[f]) cudaEventDestroy(b->ev_join[f]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_gamma) cudaEventDestroy(b->ev_gamma);
  if (b->gstream) cudaStreamDestroy(b->gstream);
  cudaFree(b->d_tiles);
  cudaFree(b->d_gent);
  cudaFree(b->d_args);
  cudaFree(b->d_counter);
  cudaFree(b->d_obs_src);
  cudaFree(b->d_obs_out);
  for (pflb_handle* h : b->dom) pflb_destroy(h);
  delete b;
  return PFLB_OK;
}

const char* pflb_batch_last_error(const pflb_batch* b) { return b ? b->err : "null batch"; }

}  // extern "C"
