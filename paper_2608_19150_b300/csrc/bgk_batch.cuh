// Batched instances: many independent problems (uneven meshes, velocity grids, nu, dt)
// advanced together.  Included at the end of bgk_lib.cu (same translation unit).
//
// Per Picard iteration the transport sweeps of all instances run as ONE persistent
// kernel: every CTA takes (instance, ordinate block) units from an atomic queue (units
// with the longest generation chains first) and splits into B sub-groups, one ordinate
// each, synchronised by named barriers.  B (ordinates per CTA; 128/B threads per
// ordinate) is the tile shape an autotuner picks per instance class by timing.  The
// small per-node kernels (Maxwellian factors, source, moments, convergence test) run as
// parallel graph branches.  One conditional while-node repeats the iteration until no
// instance is active; finished instances skip their work.

namespace bgk {

struct BatchInst {
  SweepArgs sa;
  const VGrid* g;  // device copy of the instance's velocity grid
  void* f;
  const void* src;
  const void* fbc;
  const void* Ainv;
  const DevState* ds;
  double nus;
  int type;    // 0 P1 triangle, 1 P2 triangle, 2 P1 tetrahedron, 3 Q1 parallelogram
  int B;       // ordinates per CTA
  int cached;  // local inverses available for nus
  int nv;
};

template <typename T, class E>
__device__ __noinline__ void batch_sweep_one(const BatchInst& I, int j, int tid, int nt, const NamedBarrier& bar) {
  if (I.cached)
    sweep_ordinate<E, T, true>(I.sa, *I.g, j, (T)I.nus, SrcArgs<T>{(const T*)I.src, nullptr, nullptr, T(0)},
                               (const T*)I.fbc, (const T*)I.Ainv,
                               (T*)I.f, tid, nt, bar);
  else
    sweep_ordinate<E, T, false>(I.sa, *I.g, j, (T)I.nus, SrcArgs<T>{(const T*)I.src, nullptr, nullptr, T(0)},
                                (const T*)I.fbc, nullptr, (T*)I.f, tid,
                                nt, bar);
}

// (at most 128 registers: four CTAs per SM; the dispatch's calls keep more state on the
// stack, which costs less than the residency it buys: 64-instance FP64 sweep 293 -> 252 ms)
template <typename T>
__global__ void __launch_bounds__(128, 4) k_sweep_batched(const BatchInst* __restrict__ inst,
                                                       const int2* __restrict__ units, int nunits, int* counter) {
  __shared__ int s_unit;
  for (;;) {
    if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
    __syncthreads();
    const int u = s_unit;
    __syncthreads();
    if (u >= nunits) return;
    const int2 un = units[u];
    const BatchInst& I = inst[un.x];
    if (I.ds->status != BGK_OK || I.ds->done) continue;
    const int nt = 128 / I.B;
    const int sub = threadIdx.x / nt, tid = threadIdx.x - sub * nt;
    const int j = un.y + sub;
    if (j < I.nv) {
      const NamedBarrier bar{1 + sub, nt};
      if (I.type == 1)
        batch_sweep_one<T, ElemP2Tri>(I, j, tid, nt, bar);
      else if (I.type == 0)
        batch_sweep_one<T, ElemP1Tri>(I, j, tid, nt, bar);
      else if (I.type == 3)
        batch_sweep_one<T, ElemQ1Quad>(I, j, tid, nt, bar);
      else
        batch_sweep_one<T, ElemP1Tet>(I, j, tid, nt, bar);
    }
    __syncthreads();
  }
}

// The stage loop continues while any instance is still active.
__global__ void k_any_active(DevState* const* __restrict__ ds, int n, cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int any = 0;
  for (int i = 0; i < n; ++i) any |= (ds[i]->status == BGK_OK && !ds[i]->done);
  cudaGraphSetConditional(cond, any);
}

}  // namespace bgk

struct bgk_batch {
  std::vector<bgk_handle*> inst;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int precision = BGK_FP64;
  // parallel branches of the per-node kernels: one stream pool for the step graph and one
  // for the loop body (a stream stays in a capture until that capture ends, so the two
  // captures must not share streams)
  std::vector<cudaStream_t> side_outer, side_body;
  std::vector<cudaEvent_t> ev;
  BatchInst* d_inst = nullptr;
  VGrid* d_grids = nullptr;
  int2* d_units = nullptr;
  int nunits = 0;
  int* d_counter = nullptr;
  DevState** d_ds = nullptr;
  std::vector<BatchInst> h_inst;
  // mixed precision: the instances' FP32 shadows, swept by a second batched launch
  bool mixed = false;
  BatchInst* d_inst32 = nullptr;
  DevState** d_ds32 = nullptr;
  std::vector<BatchInst> h_inst32;
  int ctas = 0;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  double sweep_ms = 0.0;
  int64_t sweep_launches = 0;
};

namespace {

// Progress messages on stderr when BGK_TRACE is set (diagnostics of the set-up path).
void trace(const char* what, int i) {
  static const bool on = std::getenv("BGK_TRACE") != nullptr;
  if (on) {
    std::fprintf(stderr, "[bgk] %s %d\n", what, i);
    std::fflush(stderr);
  }
}

int inst_type(const bgk_handle* h) { return h->hm.dim == 3 ? 2 : h->hm.quad ? 3 : (h->hm.kx == 2 ? 1 : 0); }

// Class of an instance for the autotuner: element type, velocity points, cells (log2 bucket).
uint64_t tune_key(const bgk_handle* h) {
  int lg = 0;
  while ((1 << (lg + 1)) <= h->hm.ncell) ++lg;
  return ((uint64_t)inst_type(h) << 40) | ((uint64_t)h->g.nv << 8) | (uint64_t)lg;
}

std::mutex g_tune_mutex;
std::map<uint64_t, int> g_tune_cache;  // class -> ordinates per CTA, for the process lifetime

// Unit queue: (instance, first ordinate) blocks of B ordinates, longest chains first.
int build_units(bgk_batch* b, const std::vector<int>& only) {
  std::vector<std::pair<long, int2>> u;
  for (size_t i = 0; i < b->inst.size(); ++i) {
    if (!only.empty() && std::find(only.begin(), only.end(), (int)i) == only.end()) continue;
    const bgk_handle* h = b->inst[i];
    const int B = b->h_inst[i].B;
    const long cost = (long)h->Gmax * std::max(1, h->hm.ncell / std::max(1, h->Gmax) / (128 / B) + 1);
    for (int j = 0; j < h->g.nv; j += B) u.push_back({cost, make_int2((int)i, j)});
  }
  std::stable_sort(u.begin(), u.end(), [](const std::pair<long, int2>& a, const std::pair<long, int2>& c) {
    return a.first > c.first;
  });
  std::vector<int2> flat(u.size());
  for (size_t k = 0; k < u.size(); ++k) flat[k] = u[k].second;
  b->nunits = (int)flat.size();
  if (b->d_units) cudaFree(b->d_units);
  b->d_units = nullptr;
  if (dalloc(b->d_units, sizeof(int2) * std::max<size_t>(1, flat.size())) != BGK_OK) return BGK_E_OOM;
  CK(cudaMemcpyAsync(b->d_units, flat.data(), sizeof(int2) * flat.size(), cudaMemcpyHostToDevice, b->stream));
  CK(cudaMemcpyAsync(b->d_inst, b->h_inst.data(), sizeof(BatchInst) * b->h_inst.size(), cudaMemcpyHostToDevice,
                     b->stream));
  if (b->mixed) {
    for (size_t i = 0; i < b->h_inst.size(); ++i) b->h_inst32[i].B = b->h_inst[i].B;
    CK(cudaMemcpyAsync(b->d_inst32, b->h_inst32.data(), sizeof(BatchInst) * b->h_inst32.size(),
                       cudaMemcpyHostToDevice, b->stream));
  }
  CK(cudaStreamSynchronize(b->stream));
  return BGK_OK;
}

void launch_batched_sweep(bgk_batch* b, cudaStream_t s, bool shadows = false) {
  cudaMemsetAsync(b->d_counter, 0, sizeof(int), s);
  if (shadows)
    k_sweep_batched<float><<<b->ctas, 128, 0, s>>>(b->d_inst32, b->d_units, b->nunits, b->d_counter);
  else if (b->precision == BGK_FP64)
    k_sweep_batched<double><<<b->ctas, 128, 0, s>>>(b->d_inst, b->d_units, b->nunits, b->d_counter);
  else
    k_sweep_batched<float><<<b->ctas, 128, 0, s>>>(b->d_inst, b->d_units, b->nunits, b->d_counter);
}

// Per-instance kernels of one phase on parallel branches (streams `side`) forked from
// stream s and joined back into it.
template <class F>
int fork_instances(bgk_batch* b, cudaStream_t s, const std::vector<cudaStream_t>& side, F&& body) {
  const int ns = (int)side.size();
  CK(cudaEventRecord(b->ev[0], s));
  for (int k = 0; k < ns; ++k) CK(cudaStreamWaitEvent(side[k], b->ev[0], 0));
  int rc = BGK_OK;
  for (size_t i = 0; i < b->inst.size() && rc == BGK_OK; ++i) {
    bgk_handle* h = b->inst[i];
    cudaStream_t keep = h->stream;
    h->stream = side[i % ns];
    rc = body(h);
    h->stream = keep;
  }
  for (int k = 0; k < ns; ++k) {
    CK(cudaEventRecord(b->ev[1 + k], side[k]));
    CK(cudaStreamWaitEvent(s, b->ev[1 + k], 0));
  }
  return rc;
}

// One conditional while-loop in the capture of stream s: body(bs) records the loop body
// on stream bs; the loop repeats while k_any_active(ds list) finds an active problem.
template <class F>
int batch_loop(bgk_batch* b, cudaStream_t s, DevState** d_ds, F&& body) {
  cudaGraphConditionalHandle cond = 0;
  cudaGraph_t bodyg;
  int rc = add_while(s, &cond, &bodyg);
  if (rc != BGK_OK) return rc;
  cudaStream_t bs = nullptr;
  CK(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
  if (cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess) {
    cudaStreamDestroy(bs);
    return BGK_E_CUDA;
  }
  rc = body(bs);
  if (rc == BGK_OK) k_any_active<<<1, 1, 0, bs>>>(d_ds, (int)b->inst.size(), cond);
  if (rc == BGK_OK && cudaGetLastError() != cudaSuccess) rc = BGK_E_CUDA;
  cudaGraph_t body_out = nullptr;
  if (cudaStreamEndCapture(bs, &body_out) != cudaSuccess && rc == BGK_OK) rc = BGK_E_CUDA;
  cudaStreamDestroy(bs);
  return rc;
}

// One backward-Euler step of every instance as one graph (Sec. 3.5 with S = 1).  With a
// guess attached, each instance's iterate 0 takes its guessed moments (hooks run one
// after another: instances share the network's scratch).  Mixed precision: a batched
// FP32 phase over the shadows, then the batched FP64 phase.
int capture_batch_step(bgk_batch* b) {
  cudaStream_t s = b->stream;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int rc = fork_instances(b, s, b->side_outer, [&](bgk_handle* h) {
    k_reset_state<<<1, 1, 0, h->stream>>>(h->ds);
    if (cudaMemcpyAsync(h->fk, h->f, h->nfv * h->tsize, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
      return BGK_E_CUDA;
    k_stage_begin<<<1, 1, 0, h->stream>>>(h->ds, 0);
    moments(h, 0);
    return BGK_OK;
  });
  for (size_t i = 0; i < b->inst.size() && rc == BGK_OK; ++i) {
    bgk_handle* h = b->inst[i];
    if (!h->guess) continue;
    cudaStream_t keep = h->stream;
    h->stream = s;
    rc = guess_hook(h);
    h->stream = keep;
  }
  if (rc == BGK_OK && b->mixed) {
    // FP32 phase: shadows start from the FP64 state and its (possibly guessed) moments
    rc = fork_instances(b, s, b->side_outer, [&](bgk_handle* h) {
      bgk_handle* sh = h->shadow;
      k_reset_state<<<1, 1, 0, h->stream>>>(sh->ds);
      k_stage_begin<<<1, 1, 0, h->stream>>>(sh->ds, 0);
      k_convert_gated<double, float><<<148 * 2, 256, 0, h->stream>>>(h->nfv, (const double*)h->f, (float*)sh->f,
                                                                     nullptr);
      k_convert_gated<double, float><<<148 * 2, 256, 0, h->stream>>>(h->nfv, (const double*)h->fk, (float*)sh->fk,
                                                                     nullptr);
      k_copy_moments<<<148, 256, 0, h->stream>>>((size_t)h->nnode * h->nm, h->U[0], h->U[1], h->ds, sh->U[0],
                                                 sh->U[1], sh->ds);
      return BGK_OK;
    });
    if (rc == BGK_OK)
      rc = batch_loop(b, s, b->d_ds32, [&](cudaStream_t bs) {
        int r = fork_instances(b, bs, b->side_body, [&](bgk_handle* h) {
          bgk_handle* sh = h->shadow;
          cudaStream_t keep = sh->stream;
          sh->stream = h->stream;
          const int rr = build_src_shadow(sh, (const float*)sh->fk, h->qscale_main);
          sh->stream = keep;
          return rr;
        });
        if (r == BGK_OK) launch_batched_sweep(b, bs, true);
        if (r == BGK_OK)
          r = fork_instances(b, bs, b->side_body, [&](bgk_handle* h) {
            bgk_handle* sh = h->shadow;
            cudaStream_t keep = sh->stream;
            sh->stream = h->stream;
            moments(sh, 1);
            sh->stream = keep;
            const double tol = h->cfg.tau / std::max(1.0, h->phys.nu * h->dt);
            k_finalize<<<1, 256, 0, h->stream>>>(sh->ds, sh->partial, sh->mom_blocks, std::max(tol, h->fp32_floor),
                                                 sh->cfg.l_max, 0, 0, 0, 1, tol);
            return BGK_OK;
          });
        return r;
      });
    if (rc == BGK_OK)
      rc = fork_instances(b, s, b->side_outer, [&](bgk_handle* h) {
        bgk_handle* sh = h->shadow;
        k_record_fp32<<<1, 1, 0, h->stream>>>(sh->ds, h->ds, 0);
        k_convert_gated<float, double><<<148 * 2, 256, 0, h->stream>>>(h->nfv, (const float*)sh->f, (double*)h->f,
                                                                       sh->ds);
        moments(h, 0);
        return BGK_OK;
      });
  }
  if (rc == BGK_OK)
    rc = batch_loop(b, s, b->d_ds, [&](cudaStream_t bs) {
      int r = fork_instances(b, bs, b->side_body, [&](bgk_handle* h) { return build_src(h, h->fk, h->qscale_main, h->nus_main); });
      if (r == BGK_OK) launch_batched_sweep(b, bs);
      if (r == BGK_OK)
        r = fork_instances(b, bs, b->side_body, [&](bgk_handle* h) {
          moments(h, 1);
          const double tol = h->cfg.tau / std::max(1.0, h->phys.nu * h->dt);
          k_finalize<<<1, 256, 0, h->stream>>>(h->ds, h->partial, h->mom_blocks, tol, h->cfg.l_max, 0, 0, 0);
          return BGK_OK;
        });
      return r;
    });
  if (cudaStreamEndCapture(s, &graph) != cudaSuccess && rc == BGK_OK) rc = BGK_E_CUDA;
  cudaGetLastError();
  if (rc != BGK_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  cudaError_t e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  return e == cudaSuccess ? BGK_OK : BGK_E_CUDA;
}

void release_batch(bgk_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (bgk_handle* h : b->inst) release(h);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaStream_t x : b->side_outer)
    if (x) cudaStreamDestroy(x);
  for (cudaStream_t x : b->side_body)
    if (x) cudaStreamDestroy(x);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  if (b->t0) cudaEventDestroy(b->t0);
  if (b->t1) cudaEventDestroy(b->t1);
  void* ptrs[] = {b->d_inst, b->d_grids, b->d_units, b->d_counter, b->d_ds, b->d_inst32, b->d_ds32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// Time the batched sweep of the instances in `only` with their current B (median of reps).
int time_batched_sweep(bgk_batch* b, const std::vector<int>& only, int reps, float* ms_out) {
  int rc = build_units(b, only);
  if (rc != BGK_OK) return rc;
  std::vector<float> t;
  for (int r = 0; r < reps; ++r) {
    CK(cudaEventRecord(b->t0, b->stream));
    launch_batched_sweep(b, b->stream);
    CK(cudaEventRecord(b->t1, b->stream));
    CK(cudaEventSynchronize(b->t1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, b->t0, b->t1));
    t.push_back(ms);
  }
  std::sort(t.begin(), t.end());
  *ms_out = t[t.size() / 2];
  return BGK_OK;
}

}  // namespace

extern "C" {

int bgk_batch_create(int n, const bgk_mesh* meshes, const bgk_vgrid* vgrids, const bgk_physics* phys,
                     const bgk_config* cfg, bgk_batch** out) {
  if (n <= 0 || !meshes || !vgrids || !phys || !out) return BGK_E_INVALID;
  *out = nullptr;
  bgk_batch* b = new (std::nothrow) bgk_batch();
  if (!b) return BGK_E_OOM;
  bgk_config c = cfg ? *cfg : bgk_config{};
  b->precision = c.precision == BGK_FP32_SWEEP ? BGK_FP32_SWEEP : BGK_FP64;
  b->mixed = c.precision == BGK_MIXED;
  if (c.stream) {
    b->stream = (cudaStream_t)c.stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return BGK_E_CUDA;
    }
    b->own_stream = true;
  }
  c.stream = b->stream;
  c.eager = 1;  // instances never capture their own graphs; the batch captures one
  c.sweep_front = 2;  // the batched sweep reads upwind traces from global memory
  c.hp_sweep = 1;  // the batched sweep runs FP64 data in FP64 arithmetic
  const int cache_policy = c.cache_inverse;
  c.cache_inverse = 2;  // caches are added below, once every instance's arrays exist
  for (int i = 0; i < n; ++i) {
    if (phys[i].integrator != BGK_BE) {
      release_batch(b);
      return BGK_E_INVALID;
    }
    bgk_handle* h = nullptr;
    trace("create instance", i);
    int rc = bgk_create(&meshes[i], &vgrids[i], &phys[i], &c, &h);
    if (rc != BGK_OK) {
      release_batch(b);
      return rc;
    }
    // the batched sweep reads a precomputed src (forming it in the batched sweep, as the
    // single-problem FP32 sweep does, made the 64-instance FP32 sweep 94 -> 118 ms)
    h->fuse_src = false;
    if (h->shadow) h->shadow->fuse_src = false;
    b->inst.push_back(h);
  }
  const int ns = std::min(8, n);
  b->side_outer.assign(ns, nullptr);
  b->side_body.assign(ns, nullptr);
  b->ev.resize(ns + 1);
  int rc = BGK_OK;
  for (int k = 0; k < ns; ++k)
    if (cudaStreamCreateWithFlags(&b->side_outer[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->side_body[k], cudaStreamNonBlocking) != cudaSuccess)
      rc = BGK_E_CUDA;
  for (auto& e : b->ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = BGK_E_CUDA;
  if (cudaEventCreate(&b->t0) != cudaSuccess || cudaEventCreate(&b->t1) != cudaSuccess) rc = BGK_E_CUDA;
  if (rc == BGK_OK) rc = dalloc(b->d_inst, sizeof(BatchInst) * n);
  if (rc == BGK_OK) rc = dalloc(b->d_grids, sizeof(VGrid) * n);
  if (rc == BGK_OK) rc = dalloc(b->d_counter, sizeof(int));
  if (rc == BGK_OK) rc = dalloc(b->d_ds, sizeof(DevState*) * n);
  if (rc != BGK_OK) {
    release_batch(b);
    return rc;
  }
  // local-inverse caches, largest instances first, while the policy allows
  if (cache_policy != 2) {
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int c2) { return b->inst[a]->nfv > b->inst[c2]->nfv; });
    for (int i : order) {
      bgk_handle* h = b->inst[i];
      h->cfg.cache_inverse = cache_policy;
      rc = build_inverse_cache(h, h->nus_main);
      if (rc != BGK_OK) {
        release_batch(b);
        return rc;
      }
    }
    cudaStreamSynchronize(b->stream);
  }
  std::vector<DevState*> dsp(n);
  b->h_inst.resize(n);
  for (int i = 0; i < n; ++i) {
    bgk_handle* h = b->inst[i];
    cudaMemcpyAsync(b->d_grids + i, &h->g, sizeof(VGrid), cudaMemcpyHostToDevice, b->stream);
    BatchInst I;
    I.sa = sweep_args(h);
    I.g = b->d_grids + i;
    I.f = h->f;
    I.src = h->src;
    I.fbc = h->fbc;
    I.Ainv = h->Ainv;
    I.ds = h->ds;
    I.nus = h->nus_main;
    I.type = inst_type(h);
    I.cached = h->Ainv && h->nus_cached == h->nus_main;
    I.nv = h->g.nv;
    // default tile: one ordinate per CTA when generations are wide, more when narrow
    const int width = h->hm.ncell / std::max(1, h->Gmax);
    I.B = width >= 96 ? 1 : (width >= 48 ? 2 : 4);
    b->h_inst[i] = I;
    dsp[i] = h->ds;
  }
  cudaMemcpyAsync(b->d_ds, dsp.data(), sizeof(DevState*) * n, cudaMemcpyHostToDevice, b->stream);
  if (b->mixed) {
    // the shadows' descriptors: same grids and schedules, FP32 state, no inverse cache
    if (dalloc(b->d_inst32, sizeof(BatchInst) * n) != BGK_OK || dalloc(b->d_ds32, sizeof(DevState*) * n) != BGK_OK) {
      release_batch(b);
      return BGK_E_OOM;
    }
    b->h_inst32 = b->h_inst;
    std::vector<DevState*> ds32(n);
    for (int i = 0; i < n; ++i) {
      bgk_handle* sh = b->inst[i]->shadow;
      BatchInst& I = b->h_inst32[i];
      I.sa = sweep_args(sh);
      I.f = sh->f;
      I.src = sh->src;
      I.fbc = sh->fbc;
      I.Ainv = sh->Ainv;
      I.ds = sh->ds;
      I.nus = sh->nus_main;
      I.cached = sh->Ainv && sh->nus_cached == sh->nus_main;
      ds32[i] = sh->ds;
    }
    cudaMemcpyAsync(b->d_ds32, ds32.data(), sizeof(DevState*) * n, cudaMemcpyHostToDevice, b->stream);
  }
  int per_sm = 0;
  if (b->precision == BGK_FP64)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_batched<double>, 128, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_batched<float>, 128, 0);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->ctas = std::max(1, per_sm) * sms;
  trace("units", (int)n);
  rc = build_units(b, {});
  trace("capture", rc);
  if (rc == BGK_OK) rc = capture_batch_step(b);
  trace("captured", rc);
  if (rc != BGK_OK) {
    release_batch(b);
    return rc;
  }
  *out = b;
  return BGK_OK;
}

int bgk_batch_destroy(bgk_batch* b) {
  release_batch(b);
  return BGK_OK;
}

int bgk_batch_instance(bgk_batch* b, int i, bgk_handle** h) {
  if (!b || !h || i < 0 || i >= (int)b->inst.size()) return BGK_E_INVALID;
  *h = b->inst[i];
  return BGK_OK;
}

int bgk_batch_autotune(bgk_batch* b, int reps, int32_t* h_block) {
  if (!b) return BGK_E_INVALID;
  if (reps <= 0) reps = 3;
  // group instances by class; time each candidate tile shape on the whole class
  std::map<uint64_t, std::vector<int>> cls;
  for (size_t i = 0; i < b->inst.size(); ++i) cls[tune_key(b->inst[i])].push_back((int)i);
  for (auto& kv : cls) {
    int best = -1;
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      auto it = g_tune_cache.find(kv.first);
      if (it != g_tune_cache.end()) best = it->second;
    }
    if (best < 0) {
      // the timing sweeps overwrite f: save and restore it (not needed before any state
      // has been set, which is when a caller short of memory should tune)
      std::vector<void*> saved;
      for (int i : kv.second) {
        bgk_handle* h = b->inst[i];
        void* p = nullptr;
        if (h->state_set) {
          if (dalloc(p, h->nfv * h->tsize) != BGK_OK) return BGK_E_OOM;
          cudaMemcpyAsync(p, h->f, h->nfv * h->tsize, cudaMemcpyDeviceToDevice, b->stream);
        }
        saved.push_back(p);
        k_reset_state<<<1, 1, 0, b->stream>>>(h->ds);
      }
      float best_ms = 1e30f;
      for (int B : {1, 2, 4}) {
        for (int i : kv.second) b->h_inst[i].B = B;
        float ms = 0.f;
        int rc = time_batched_sweep(b, kv.second, reps, &ms);
        if (rc != BGK_OK) return rc;
        if (ms < best_ms) {
          best_ms = ms;
          best = B;
        }
      }
      for (size_t k = 0; k < kv.second.size(); ++k) {
        bgk_handle* h = b->inst[kv.second[k]];
        if (saved[k])
          cudaMemcpyAsync(h->f, saved[k], h->nfv * h->tsize, cudaMemcpyDeviceToDevice, b->stream);
        else
          cudaMemsetAsync(h->f, 0, h->nfv * h->tsize, b->stream);
      }
      CK(cudaStreamSynchronize(b->stream));
      for (void* p : saved)
        if (p) cudaFree(p);
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      g_tune_cache[kv.first] = best;
    }
    for (int i : kv.second) b->h_inst[i].B = best;
  }
  if (h_block)
    for (size_t i = 0; i < b->inst.size(); ++i) h_block[i] = b->h_inst[i].B;
  int rc = build_units(b, {});
  if (rc == BGK_OK) rc = capture_batch_step(b);
  return rc;
}

int bgk_batch_set_guess(bgk_batch* b, bgk_mlp* m) {
  if (!b) return BGK_E_INVALID;
  CK(cudaStreamSynchronize(b->stream));
  for (bgk_handle* h : b->inst) {
    if (m && (m->F != guess_features(h->hm.dim) || m->O != h->nm)) return BGK_E_INVALID;
    if (m) {
      int rc = guess_buffers(h);
      if (rc == BGK_OK) rc = mlp_reserve(m, std::max<int64_t>(m->cap, h->nnode));
      if (rc != BGK_OK) return rc;
    }
    h->guess = m;
  }
  if (m) {
    k_to_bf16<<<(m->np + 255) / 256, 256, 0, b->stream>>>(m->np, m->p, m->pb);
    m->pb_valid = true;
  }
  CK(cudaStreamSynchronize(b->stream));
  return capture_batch_step(b);
}

int bgk_batch_step(bgk_batch* b, int nsteps, int32_t* h_iters, int32_t* h_status) {
  if (!b || nsteps < 0) return BGK_E_INVALID;
  for (int k = 0; k < nsteps; ++k) CK(cudaGraphLaunch(b->exec, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  int worst = BGK_OK;
  for (size_t i = 0; i < b->inst.size(); ++i) {
    DevState d;
    CK(cudaMemcpy(&d, b->inst[i]->ds, sizeof(DevState), cudaMemcpyDeviceToHost));
    if (h_iters) h_iters[i] = d.iters[0] + d.iters32[0];
    if (h_status) h_status[i] = d.status;
    if (d.status != BGK_OK && worst == BGK_OK) worst = d.status;
  }
  return worst;
}

int bgk_batch_sweep(bgk_batch* b) {
  if (!b) return BGK_E_INVALID;
  for (bgk_handle* h : b->inst) {
    cudaStream_t keep = h->stream;
    h->stream = b->stream;
    k_reset_state<<<1, 1, 0, b->stream>>>(h->ds);
    moments(h, 0);
    int rc = build_src(h, h->fk, h->qscale_main, h->nus_main);
    h->stream = keep;
    if (rc != BGK_OK) return rc;
  }
  CK(cudaEventRecord(b->t0, b->stream));
  launch_batched_sweep(b, b->stream);
  CK(cudaEventRecord(b->t1, b->stream));
  CK(cudaEventSynchronize(b->t1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, b->t0, b->t1));
  b->sweep_ms += ms;
  b->sweep_launches += 1;
  return BGK_OK;
}

int bgk_batch_info(const bgk_batch* b, int64_t* out) {
  if (!b || !out) return BGK_E_INVALID;
  int64_t dof = 0;
  for (const bgk_handle* h : b->inst) dof += (int64_t)h->nfv;
  out[0] = (int64_t)b->inst.size();
  out[1] = dof;
  out[2] = b->nunits;
  out[3] = b->ctas;
  return BGK_OK;
}

int bgk_batch_timing(bgk_batch* b, int reset, double* sweep_ms_total, int64_t* sweep_launches) {
  if (!b) return BGK_E_INVALID;
  if (sweep_ms_total) *sweep_ms_total = b->sweep_ms;
  if (sweep_launches) *sweep_launches = b->sweep_launches;
  if (reset) {
    b->sweep_ms = 0.0;
    b->sweep_launches = 0;
  }
  return BGK_OK;
}

}  // extern "C"
