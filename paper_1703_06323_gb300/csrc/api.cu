// C ABI of libufe (declarations and contracts in include/ufe.h).
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>

#include "bddc.cuh"

struct ufe_mesh : ufe::Mesh {};
struct ufe_system : ufe::System {};
struct ufe_bddc : ufe::Bddc {};

namespace ufe {

static thread_local std::string g_last_error;
std::atomic<long long> g_kernel_launches{0};
thread_local long long* g_capture_counter = nullptr;

// ---- kernel timing -------------------------------------------------------------
namespace {
std::mutex g_tmu;
bool g_timing = false;
struct TRec {
  std::string name;
  cudaEvent_t e0, e1;
};
std::vector<TRec> g_trecs;
}  // namespace

void TimedLaunch::begin(const char* nm, cudaStream_t s) {
  if (!g_timing || g_capture_counter) return;   // never inside a graph capture
  name = nm;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
}

void TimedLaunch::end(cudaStream_t s) {
  if (!e0) return;
  cudaEventRecord(e1, s);
  std::lock_guard<std::mutex> lock(g_tmu);
  g_trecs.push_back({name, e0, e1});
  e0 = e1 = nullptr;
}

void note_launch() {
  if (g_capture_counter)
    ++*g_capture_counter;
  else
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
}

void set_error(const std::string& msg) { g_last_error = msg; }

void copy_in(void* dst_dev, const void* src, size_t bytes, int mem, cudaStream_t s) {
  if (!bytes) return;
  UFE_CUDA(cudaMemcpyAsync(dst_dev, src, bytes, mem == UFE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           s));
}

void copy_out(void* dst, const void* src_dev, size_t bytes, int mem, cudaStream_t s) {
  if (!bytes) return;
  UFE_CUDA(cudaMemcpyAsync(dst, src_dev, bytes, mem == UFE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           s));
  UFE_CUDA(cudaStreamSynchronize(s));
}

template <typename F>
static ufe_status guarded(F f) {
  try {
    f();
    g_last_error.clear();
    return UFE_OK;
  } catch (const Error& e) {
    g_last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return UFE_ERR_OUT_OF_MEMORY;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return UFE_ERR_INVALID_ARG;
  }
}

static void check_mem(int mem) {
  UFE_REQUIRE(mem == UFE_MEM_HOST || mem == UFE_MEM_DEVICE, UFE_ERR_INVALID_ARG, "mem must be UFE_MEM_HOST or UFE_MEM_DEVICE");
}

// device copy of an optional input array (nullptr stays nullptr)
template <typename T>
static const T* stage(DBuf<T>& buf, const T* src, size_t n, int mem, cudaStream_t s) {
  if (!src) return nullptr;
  if (mem == UFE_MEM_DEVICE) return src;
  buf.alloc(n, s);
  copy_in(buf.p, src, n * sizeof(T), mem, s);
  return buf.p;
}

// The library's buffers are stream-ordered allocations from the device's default memory
// pool.  With the pool's default release threshold (0) every synchronisation returns the
// freed memory to the driver and the next set-up maps it again; a threshold of the whole
// device keeps it cached in the pool for reuse (once per device, process-local).
void keep_pool_memory() {
  static std::mutex mu;
  static bool done[128] = {};
  int dev = 0;
  UFE_CUDA(cudaGetDevice(&dev));
  UFE_REQUIRE(dev >= 0 && dev < 128, UFE_ERR_UNSUPPORTED, "device ordinal beyond 127");
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  UFE_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t keep = UINT64_MAX;
  UFE_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  done[dev] = true;
}

// FMA-rate probe: eight independent chains per thread keep every pipe slot busy
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T* out) {
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = T(threadIdx.x + i) * T(1e-3);
  const T b = T(0.999999), c = T(1e-7);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  }
  T sum = T(0);
#pragma unroll
  for (int i = 0; i < 8; ++i) sum += a[i];
  if (sum == T(-1.2345)) out[0] = sum;   // keeps the chains live; never true
}

bool timing_enabled() { return g_timing; }
void set_timing_enabled(bool on) { g_timing = on; }

}  // namespace ufe

using namespace ufe;

extern "C" {

const char* ufe_last_error(void) { return g_last_error.c_str(); }

int ufe_version(void) { return 100; }

int64_t ufe_kernel_launches(void) { return (int64_t)g_kernel_launches.load(); }

void ufe_timing_enable(int on) { g_timing = on != 0; }

ufe_status ufe_probe_fma_rate(int kind, void* stream, double* tflops) {
  return guarded([&] {
    UFE_REQUIRE(tflops && (kind == 0 || kind == 1), UFE_ERR_INVALID_ARG, "bad probe arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    UFE_CUDA(cudaGetDevice(&dev));
    UFE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = 4u * (unsigned)sms;
    // a few milliseconds per launch on GB300 (about 1.2 TFLOP/s FP64, 70 TFLOP/s FP32)
    const int iters = kind == 0 ? 4000 : 200000;
    DBuf<double> out;
    out.alloc(1, s);
    cudaEvent_t e0, e1;
    UFE_CUDA(cudaEventCreate(&e0));
    UFE_CUDA(cudaEventCreate(&e1));
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
      UFE_CUDA(cudaEventRecord(e0, s));
      if (kind == 0)
        k_fma_probe<double><<<grid, 256, 0, s>>>(iters, out.p);
      else
        k_fma_probe<float><<<grid, 256, 0, s>>>(iters, reinterpret_cast<float*>(out.p));
      UFE_CHECK_LAUNCH();
      UFE_CUDA(cudaEventRecord(e1, s));
      UFE_CUDA(cudaEventSynchronize(e1));
      UFE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * 8.0 * (double)iters * grid * 256.0;
    *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
  });
}

void ufe_timing_reset(void) {
  std::lock_guard<std::mutex> lock(g_tmu);
  for (auto& r : g_trecs) {
    cudaEventSynchronize(r.e1);
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  g_trecs.clear();
}

ufe_status ufe_timing_get(const char* kernel, double* total_ms, int64_t* launches) {
  return guarded([&] {
    UFE_REQUIRE(kernel && total_ms && launches, UFE_ERR_INVALID_ARG, "null argument");
    const std::string k(kernel);
    static const char* known[] = {"gj_update_f64", "gj_update_f32", "integrate_cut", "phase_mesh",
                                  "phase_assemble", "phase_objects", "phase_local", "phase_factor",
                                  "phase_coarse", "phase_solve", "apply", "prec_interior",
                                  "prec_neumann", "coarse_solve", "prec_prolong", "prec_final",
                                  "gj_diag_f64", "gj_diag_f32", "gj_panel_f64", "gj_panel_f32",
                                  "gj_lookahead_f64", "gj_lookahead_f32"};
    bool ok = false;
    for (const char* kn : known) ok = ok || k == kn;
    UFE_REQUIRE(ok, UFE_ERR_INVALID_ARG, "unknown timed kernel or phase");
    std::lock_guard<std::mutex> lock(g_tmu);
    double tot = 0.0;
    int64_t n = 0;
    for (auto& r : g_trecs) {
      if (r.name != k) continue;
      UFE_CUDA(cudaEventSynchronize(r.e1));
      float ms = 0.f;
      UFE_CUDA(cudaEventElapsedTime(&ms, r.e0, r.e1));
      tot += ms;
      ++n;
    }
    *total_ms = tot;
    *launches = n;
  });
}

ufe_status ufe_mesh_create(const double box_lo[3], const double box_hi[3], const int32_t cells[3],
                           const int32_t sub_cells[3], const double* phi_nodes, int mem, uint32_t dirichlet_face_mask,
                           int64_t pin_node, void* stream, ufe_mesh** out) {
  return guarded([&] {
    UFE_REQUIRE(box_lo && box_hi && cells && sub_cells && phi_nodes && out, UFE_ERR_INVALID_ARG, "null argument");
    check_mem(mem);
    *out = nullptr;
    keep_pool_memory();
    std::unique_ptr<ufe_mesh> m(new ufe_mesh());
    m->stream = (cudaStream_t)stream;
    GridGeom& g = m->g;
    g.nx = cells[0]; g.ny = cells[1]; g.nz = cells[2];
    g.sx = sub_cells[0]; g.sy = sub_cells[1]; g.sz = sub_cells[2];
    UFE_REQUIRE(g.nx > 0 && g.ny > 0 && g.nz > 0, UFE_ERR_INVALID_ARG, "cells must be positive");
    UFE_REQUIRE(g.sx >= 1 && g.sy >= 1 && g.sz >= 1 && g.sx <= 16 && g.sy <= 16 && g.sz <= 16, UFE_ERR_INVALID_ARG,
                "sub_cells must lie in 1..16");
    UFE_REQUIRE(g.nx % g.sx == 0 && g.ny % g.sy == 0 && g.nz % g.sz == 0, UFE_ERR_INVALID_ARG,
                "sub_cells must divide cells");
    UFE_REQUIRE((int64_t)(g.nx + 1) * (g.ny + 1) * (g.nz + 1) < (int64_t)1 << 31, UFE_ERR_INVALID_ARG, "grid too large");
    UFE_REQUIRE(dirichlet_face_mask < 64, UFE_ERR_INVALID_ARG, "dirichlet_face_mask has bits beyond the 6 faces");
    double hs[3];
    for (int d = 0; d < 3; ++d) {
      UFE_REQUIRE(box_hi[d] > box_lo[d], UFE_ERR_INVALID_ARG, "empty box");
      g.lo[d] = box_lo[d];
      hs[d] = (box_hi[d] - box_lo[d]) / cells[d];
    }
    UFE_REQUIRE(std::fabs(hs[0] - hs[1]) <= 1e-12 * hs[0] && std::fabs(hs[0] - hs[2]) <= 1e-12 * hs[0],
                UFE_ERR_INVALID_ARG, "cells must be cubes");
    g.h = hs[0];
    g.bx = g.nx / g.sx; g.by = g.ny / g.sy; g.bz = g.nz / g.sz;
    g.lnx = g.sx + 1; g.lny = g.sy + 1; g.lnz = g.sz + 1;
    g.n_local_nodes = g.lnx * g.lny * g.lnz;
    m->face_mask = dirichlet_face_mask;
    const int64_t nn = g.n_nodes();
    m->phi.alloc(nn, m->stream);
    copy_in(m->phi.p, phi_nodes, nn * sizeof(double), mem, m->stream);
    TimedLaunch tl;
    tl.begin("phase_mesh", m->stream);
    mesh_build(*m, m->phi.p, pin_node);
    tl.end(m->stream);
    UFE_CUDA(cudaStreamSynchronize(m->stream));
    *out = m.release();
  });
}

ufe_status ufe_mesh_get_info(const ufe_mesh* m, ufe_mesh_info* info) {
  return guarded([&] {
    UFE_REQUIRE(m && info, UFE_ERR_INVALID_ARG, "null argument");
    info->n_nodes = m->g.n_nodes();
    info->n_cells = m->g.n_cells();
    info->n_active_cells = m->n_active;
    info->n_cut_cells = m->n_cut;
    info->n_dof = m->n_dof;
    info->n_subdomains = m->n_sub;
    info->n_interface_dofs = m->n_gamma;
    info->pinned_node = m->pin;
    info->n_constrained = m->n_constrained;
    info->max_interior = m->max_nI;
    info->max_interface = m->max_nG;
  });
}

ufe_status ufe_mesh_get_cell_types(const ufe_mesh* m, uint8_t* out, int mem) {
  return guarded([&] {
    UFE_REQUIRE(m && out, UFE_ERR_INVALID_ARG, "null argument");
    check_mem(mem);
    copy_out(out, m->cell_type.p, m->g.n_cells(), mem, m->stream);
  });
}

ufe_status ufe_mesh_get_dof_map(const ufe_mesh* m, int32_t* out, int mem) {
  return guarded([&] {
    UFE_REQUIRE(m && out, UFE_ERR_INVALID_ARG, "null argument");
    check_mem(mem);
    copy_out(out, m->dof_of_node.p, m->g.n_nodes() * 4, mem, m->stream);
  });
}

ufe_status ufe_mesh_get_subdomains(const ufe_mesh* m, int32_t* out, int mem) {
  return guarded([&] {
    UFE_REQUIRE(m && out, UFE_ERR_INVALID_ARG, "null argument");
    check_mem(mem);
    copy_out(out, m->sub_of_cell.p, m->g.n_cells() * 4, mem, m->stream);
  });
}

ufe_status ufe_mesh_get_neighbours(const ufe_mesh* m, int32_t* out, int mem) {
  return guarded([&] {
    UFE_REQUIRE(m && out, UFE_ERR_INVALID_ARG, "null argument");
    check_mem(mem);
    copy_out(out, m->neigh.p, m->n_dof * 8 * 4, mem, m->stream);
  });
}

void ufe_mesh_destroy(ufe_mesh* m) {
  if (!m) return;
  cudaStream_t s = m->stream;
  delete m;
  cudaStreamSynchronize(s);
}

ufe_status ufe_assemble(ufe_mesh* m, const double* kappa, const double* f, const double* flux, const double* gval,
                        int mem, ufe_system** out) {
  return guarded([&] {
    UFE_REQUIRE(m && out, UFE_ERR_INVALID_ARG, "null argument");
    check_mem(mem);
    *out = nullptr;
    std::unique_ptr<ufe_system> sys(new ufe_system());
    sys->mesh = m;
    sys->stream = m->stream;
    cudaStream_t s = m->stream;
    const int64_t nn = m->g.n_nodes(), nc = m->g.n_cells();
    DBuf<double> fb, qb, gb;
    if (kappa) {
      sys->has_kappa = true;
      sys->kappa.alloc(nc, s);
      copy_in(sys->kappa.p, kappa, nc * 8, mem, s);
    }
    const double* fd = stage(fb, f, nn, mem, s);
    const double* qd = stage(qb, flux, nn * 3, mem, s);
    const double* gd = stage(gb, gval, nn, mem, s);
    TimedLaunch tl;
    tl.begin("phase_assemble", s);
    system_build(*sys, sys->has_kappa ? sys->kappa.p : nullptr, fd, qd, gd);
    tl.end(s);
    UFE_CUDA(cudaStreamSynchronize(s));
    *out = sys.release();
  });
}

ufe_status ufe_assemble_nitsche(ufe_mesh* m, const double* f, const double* gval, int mem, ufe_system** out) {
  return guarded([&] {
    UFE_REQUIRE(m && gval && out, UFE_ERR_INVALID_ARG, "null argument");
    check_mem(mem);
    *out = nullptr;
    std::unique_ptr<ufe_system> sys(new ufe_system());
    sys->mesh = m;
    sys->stream = m->stream;
    cudaStream_t s = m->stream;
    const int64_t nn = m->g.n_nodes();
    DBuf<double> fb, gb;
    const double* fd = stage(fb, f, nn, mem, s);
    const double* gd = stage(gb, gval, nn, mem, s);
    TimedLaunch tl;
    tl.begin("phase_assemble", s);
    system_build(*sys, nullptr, fd, nullptr, gd, true);
    tl.end(s);
    UFE_CUDA(cudaStreamSynchronize(s));
    *out = sys.release();
  });
}

ufe_status ufe_system_get_nitsche_beta(const ufe_system* sys, double* beta, int mem) {
  return guarded([&] {
    UFE_REQUIRE(sys && beta, UFE_ERR_INVALID_ARG, "null argument");
    UFE_REQUIRE(sys->nitsche, UFE_ERR_INVALID_ARG, "the system has no weak Dirichlet data");
    check_mem(mem);
    if (sys->mesh->n_cut > 0) copy_out(beta, sys->beta.p, sys->mesh->n_cut * 8, mem, sys->stream);
    UFE_CUDA(cudaStreamSynchronize(sys->stream));
  });
}

ufe_status ufe_system_set_kappa(ufe_system* sys, const double* kappa, int mem) {
  return guarded([&] {
    UFE_REQUIRE(sys && kappa, UFE_ERR_INVALID_ARG, "null argument");
    UFE_REQUIRE(sys->ncomp == 1, UFE_ERR_UNSUPPORTED, "ufe_system_set_kappa: Poisson systems only");
    check_mem(mem);
    cudaStream_t s = sys->stream;
    // the coefficient buffer must exist already: solves captured in CUDA graphs hold its address
    UFE_REQUIRE(sys->has_kappa, UFE_ERR_INVALID_ARG,
                "ufe_system_set_kappa: the system was assembled without a per-cell coefficient");
    const int64_t nc = sys->mesh->g.n_cells();
    copy_in(sys->kappa.p, kappa, nc * 8, mem, s);
    system_rebuild_rhs(*sys);
    UFE_CUDA(cudaStreamSynchronize(s));
  });
}

ufe_status ufe_assemble_elastic(ufe_mesh* m, double E, double nu, const double* E_scale, const double* f,
                                const double* stress, const double* gval, int mem, ufe_system** out) {
  return guarded([&] {
    UFE_REQUIRE(m && out, UFE_ERR_INVALID_ARG, "null argument");
    UFE_REQUIRE(E > 0.0 && nu > -1.0 && nu < 0.5, UFE_ERR_INVALID_ARG, "need E > 0 and -1 < nu < 1/2");
    check_mem(mem);
    *out = nullptr;
    std::unique_ptr<ufe_system> sys(new ufe_system());
    sys->mesh = m;
    sys->stream = m->stream;
    sys->ncomp = 3;
    sys->lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    sys->mu = E / (2.0 * (1.0 + nu));
    cudaStream_t s = m->stream;
    const int64_t nn = m->g.n_nodes(), nc = m->g.n_cells();
    DBuf<double> fb, sb, gb;
    if (E_scale) {
      sys->has_kappa = true;
      sys->kappa.alloc(nc, s);
      copy_in(sys->kappa.p, E_scale, nc * 8, mem, s);
    }
    const double* fd = stage(fb, f, nn * 3, mem, s);
    const double* sd = stage(sb, stress, nn * 9, mem, s);
    const double* gd = stage(gb, gval, nn * 3, mem, s);
    TimedLaunch tl;
    tl.begin("phase_assemble", s);
    system_build_elastic(*sys, sys->has_kappa ? sys->kappa.p : nullptr, fd, sd, gd);
    tl.end(s);
    UFE_CUDA(cudaStreamSynchronize(s));
    *out = sys.release();
  });
}

ufe_status ufe_system_get_info(const ufe_system* sys, int32_t* ncomp, int64_t* n) {
  return guarded([&] {
    UFE_REQUIRE(sys && ncomp && n, UFE_ERR_INVALID_ARG, "null argument");
    *ncomp = sys->ncomp;
    *n = sys->n_vec();
  });
}

ufe_status ufe_system_get_rhs(const ufe_system* sys, double* b, int mem) {
  return guarded([&] {
    UFE_REQUIRE(sys && b, UFE_ERR_INVALID_ARG, "null argument");
    check_mem(mem);
    copy_out(b, sys->b.p, sys->n_vec() * 8, mem, sys->stream);
  });
}

ufe_status ufe_system_apply(const ufe_system* sys, const double* x, double* y, int mem) {
  return guarded([&] {
    UFE_REQUIRE(sys && x && y, UFE_ERR_INVALID_ARG, "null argument");
    check_mem(mem);
    cudaStream_t s = sys->stream;
    const int64_t n = sys->n_vec();
    DBuf<double> xb, yb;
    const double* xd = stage(xb, x, n, mem, s);
    double* yd = y;
    if (mem == UFE_MEM_HOST) {
      yb.alloc(n, s);
      yd = yb.p;
    }
    system_apply(*sys, xd, yd, s);
    if (mem == UFE_MEM_HOST) copy_out(y, yd, n * 8, mem, s);
    UFE_CUDA(cudaStreamSynchronize(s));
  });
}

ufe_status ufe_system_get_cut_data(const ufe_system* sys, int32_t* cut_cells, double* K, double* load, double* eta,
                                   int mem) {
  return guarded([&] {
    UFE_REQUIRE(sys, UFE_ERR_INVALID_ARG, "null argument");
    check_mem(mem);
    const int64_t n = sys->mesh->n_cut;
    const int64_t ne = 8 * sys->ncomp;
    cudaStream_t s = sys->stream;
    if (cut_cells) copy_out(cut_cells, sys->mesh->cut_cells.p, n * 4, mem, s);
    if (K) copy_out(K, sys->K_cut.p, n * ne * ne * 8, mem, s);
    if (load) copy_out(load, sys->load_cut.p, n * ne * 8, mem, s);
    if (eta) copy_out(eta, sys->eta.p, n * 8, mem, s);
  });
}

void ufe_system_destroy(ufe_system* sys) {
  if (!sys) return;
  cudaStream_t s = sys->stream;
  delete sys;
  cudaStreamSynchronize(s);
}

ufe_status ufe_bddc_setup(ufe_system* sys, const ufe_bddc_opts* opts, ufe_bddc** out) {
  return guarded([&] {
    UFE_REQUIRE(sys && opts && out, UFE_ERR_INVALID_ARG, "null argument");
    UFE_REQUIRE(opts->weighting == UFE_WEIGHT_STIFFNESS || opts->weighting == UFE_WEIGHT_TOPOLOGICAL,
                UFE_ERR_INVALID_ARG, "bad weighting");
    UFE_REQUIRE(opts->objects == UFE_OBJECTS_STANDARD || opts->objects == UFE_OBJECTS_VARIANT1 ||
                    opts->objects == UFE_OBJECTS_VARIANT2,
                UFE_ERR_INVALID_ARG, "bad objects");
    UFE_REQUIRE(opts->objects != UFE_OBJECTS_VARIANT2 || sys->ncomp == 1, UFE_ERR_UNSUPPORTED,
                "variant-2 objects: Poisson systems only");
    UFE_REQUIRE(opts->coarse >= UFE_COARSE_C && opts->coarse <= UFE_COARSE_CEF, UFE_ERR_INVALID_ARG, "bad coarse");
    UFE_REQUIRE(opts->coarse_solver >= UFE_COARSE_SOLVER_AUTO && opts->coarse_solver <= UFE_COARSE_SOLVER_BDDC,
                UFE_ERR_INVALID_ARG, "bad coarse solver");
    UFE_REQUIRE(opts->coarse_solver != UFE_COARSE_SOLVER_BDDC || (opts->coarse_group >= 0 && opts->coarse_group <= 1024),
                UFE_ERR_INVALID_ARG, "coarse_group must lie in 0..1024");
    UFE_REQUIRE(opts->precision == UFE_PREC_FP64 || opts->precision == UFE_PREC_MIXED, UFE_ERR_INVALID_ARG,
                "bad precision");
    *out = nullptr;
    std::unique_ptr<ufe_bddc> B(new ufe_bddc());
    B->sys = sys;
    B->mesh = sys->mesh;
    B->stream = sys->stream;
    B->opts = *opts;
    B->mixed = opts->precision == UFE_PREC_MIXED;
    B->coarse_solver = opts->coarse_solver;
    if (opts->coarse_solver == UFE_COARSE_SOLVER_BDDC && opts->coarse_group > 0) B->coarse_group = opts->coarse_group;
    B->coarse_keep_corners = opts->coarse_solver == UFE_COARSE_SOLVER_BDDC && opts->coarse_keep_corners != 0;
    UFE_CUDA(cudaGetDevice(&B->device));
    bddc_build(*B);
    tune_preconditioner(*B);
    bddc_noalloc_prepare(*B);
    UFE_CUDA(cudaStreamSynchronize(B->stream));
    *out = B.release();
  });
}

ufe_status ufe_bddc_get_info(const ufe_bddc* B, ufe_bddc_info* info) {
  return guarded([&] {
    UFE_REQUIRE(B && info, UFE_ERR_INVALID_ARG, "null argument");
    info->n_objects = B->n_obj;
    info->n_corners = B->n_corner;
    info->n_edges = B->n_edge;
    info->n_faces = B->n_face;
    info->n_coarse = B->n_coarse;
    info->max_local_coarse = B->max_nC;
    info->setup_ms = B->setup_ms;
    info->inverse_flops_local = B->inv_flops_local;
    info->inverse_flops_coarse = B->inv_flops_coarse;
    info->bytes_interior_inverse = B->bytes_II;
    info->bytes_neumann = B->bytes_GG;
    info->bytes_coarse_basis = B->bytes_GC;
    info->bytes_offdiag = B->bytes_off;
    info->bytes_coarse_inverse = B->bytes_Ac;
    info->interior_slots = B->n_vIloc;
    info->interface_slots = B->n_vGloc;
    info->fp64_refactor = B->fp64_refactor;
    info->coarse_solver = B->ml.n2 > 0     ? UFE_COARSE_SOLVER_BDDC
                          : B->coarse_dense ? UFE_COARSE_SOLVER_DENSE
                                            : UFE_COARSE_SOLVER_CR;
    info->level2_subdomains = B->ml.n2;
    info->level3_coarse = B->ml.n3;
    info->coarse_layers = B->cr.nlayers;
    info->cphi_error = B->cphi_error;
    info->local_tensor_cores = B->local_tc;
    info->prec_cluster = B->prec_cl;
    info->prec_stages = B->prec_stages;
    info->fp64_subdomains = B->fp64_refactor ? (int32_t)B->mesh->n_sub : (B->mixed ? B->n_sub64 : 0);
    info->coarse_levels = B->cr.nlevels;
  });
}

ufe_status ufe_bddc_get_objects(const ufe_bddc* B, int32_t* object_of_dof, int32_t* object_kind,
                                int32_t* coarse_of_object, int mem) {
  return guarded([&] {
    UFE_REQUIRE(B, UFE_ERR_INVALID_ARG, "null argument");
    check_mem(mem);
    cudaStream_t s = B->stream;
    if (object_of_dof) copy_out(object_of_dof, B->obj_of_dof.p, B->mesh->n_dof * 4, mem, s);
    if (object_kind) copy_out(object_kind, B->obj_kind.p, B->n_obj * 4, mem, s);
    if (coarse_of_object) copy_out(coarse_of_object, B->coarse_of_obj.p, B->n_obj * 4, mem, s);
  });
}

ufe_status ufe_bddc_apply(ufe_bddc* B, const double* r, double* z, int mem) {
  return guarded([&] {
    UFE_REQUIRE(B && r && z, UFE_ERR_INVALID_ARG, "null argument");
    check_mem(mem);
    cudaStream_t s = B->stream;
    const int64_t n = B->sys->n_vec();
    DBuf<double> rb, zb;
    const double* rd = stage(rb, r, n, mem, s);
    double* zd = z;
    if (mem == UFE_MEM_HOST) {
      zb.alloc(n, s);
      zd = zb.p;
    }
    UFE_CUDA(cudaMemsetAsync(zd, 0, n * 8, s));
    bddc_apply(*B, rd, zd);
    if (mem == UFE_MEM_HOST) copy_out(z, zd, n * 8, mem, s);
    UFE_CUDA(cudaStreamSynchronize(s));
  });
}

ufe_status ufe_bddc_apply_noalloc(ufe_bddc* B, const double* r_dev, double* z_dev) {
  return guarded([&] {
    UFE_REQUIRE(B && r_dev && z_dev, UFE_ERR_INVALID_ARG, "null argument");
    bddc_apply_noalloc(*B, r_dev, z_dev);
    UFE_CUDA(cudaStreamSynchronize(B->stream));
  });
}

void ufe_bddc_destroy(ufe_bddc* B) {
  if (!B) return;
  cudaStream_t s = B->stream;
  delete B;
  cudaStreamSynchronize(s);
}

ufe_status ufe_pcg_solve(ufe_system* sys, ufe_bddc* B, const double* b, double* x, int mem, const ufe_solve_opts* opts,
                         ufe_solve_info* info) {
  return guarded([&] {
    UFE_REQUIRE(sys && B && x && opts, UFE_ERR_INVALID_ARG, "null argument");
    UFE_REQUIRE(B->sys == sys, UFE_ERR_INVALID_ARG, "preconditioner belongs to another system");
    UFE_REQUIRE(opts->rtol > 0 && opts->maxit >= 0, UFE_ERR_INVALID_ARG, "bad solve options");
    check_mem(mem);
    cudaStream_t s = sys->stream;
    const int64_t n = sys->n_vec();
    DBuf<double> bb, xb;
    const double* bd = b ? stage(bb, b, n, mem, s) : sys->b.p;
    double* xd = x;
    if (mem == UFE_MEM_HOST) {
      xb.alloc(n, s);
      copy_in(xb.p, x, n * 8, mem, s);
      xd = xb.p;
    }
    struct Out {
      double* dst;
      double* src;
      int64_t n;
      int mem;
      cudaStream_t s;
      ~Out() {
        if (mem == UFE_MEM_HOST) {
          cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDeviceToHost, s);
          cudaStreamSynchronize(s);
        }
      }
    } out_guard{x, xd, n, mem, s};
    TimedLaunch tl;
    tl.begin("phase_solve", s);
    pcg_solve(*B, bd, xd, *opts, info);
    tl.end(s);
  });
}

ufe_status ufe_pcg_solve_batched(int32_t n, ufe_system* const* systems, ufe_bddc* const* bddcs, const double* const* b,
                                 double* const* x, int mem, const ufe_solve_opts* opts, ufe_solve_info* infos) {
  ufe_status result = UFE_OK;
  const ufe_status st = guarded([&] {
    UFE_REQUIRE(n >= 0, UFE_ERR_INVALID_ARG, "negative problem count");
    if (n == 0) return;
    UFE_REQUIRE(systems && bddcs && x && opts, UFE_ERR_INVALID_ARG, "null argument");
    UFE_REQUIRE(opts->rtol > 0 && opts->maxit >= 0, UFE_ERR_INVALID_ARG, "bad solve options");
    check_mem(mem);
    std::vector<Bddc*> Bs(n);
    for (int i = 0; i < n; ++i) {
      UFE_REQUIRE(systems[i] && bddcs[i] && x[i], UFE_ERR_INVALID_ARG, "null problem " + std::to_string(i));
      UFE_REQUIRE(bddcs[i]->sys == systems[i], UFE_ERR_INVALID_ARG,
                  "preconditioner " + std::to_string(i) + " belongs to another system");
      for (int j = 0; j < i; ++j)
        UFE_REQUIRE(bddcs[j] != bddcs[i], UFE_ERR_INVALID_ARG, "a preconditioner appears twice in the batch");
      Bs[i] = bddcs[i];
    }
    std::vector<DBuf<double>> bb(n), xb(n);
    std::vector<const double*> bd(n);
    std::vector<double*> xd(n);
    for (int i = 0; i < n; ++i) {
      cudaStream_t s = systems[i]->stream;
      const int64_t len = systems[i]->n_vec();
      bd[i] = (b && b[i]) ? stage(bb[i], b[i], len, mem, s) : systems[i]->b.p;
      xd[i] = x[i];
      if (mem == UFE_MEM_HOST) {
        xb[i].alloc(len, s);
        copy_in(xb[i].p, x[i], len * 8, mem, s);
        xd[i] = xb[i].p;
      }
    }
    result = pcg_solve_batched(n, Bs.data(), bd.data(), xd.data(), *opts, infos);
    if (mem == UFE_MEM_HOST)
      for (int i = 0; i < n; ++i) copy_out(x[i], xd[i], systems[i]->n_vec() * 8, mem, systems[i]->stream);
  });
  if (st != UFE_OK) return st;
  if (result == UFE_ERR_BREAKDOWN) set_error("PCG breakdown (p.Ap <= 0) in at least one problem of the batch");
  if (result == UFE_ERR_NO_CONVERGENCE) set_error("at least one problem of the batch did not reach the tolerance");
  return result;
}

ufe_status ufe_adjoint(ufe_system* sys, ufe_bddc* B, const double* u, const double* dJdu, double* lambda,
                       double* dJdkappa, int mem, const ufe_solve_opts* opts, ufe_solve_info* info) {
  return guarded([&] {
    UFE_REQUIRE(sys && B && u && dJdu && lambda && dJdkappa && opts, UFE_ERR_INVALID_ARG, "null argument");
    UFE_REQUIRE(B->sys == sys, UFE_ERR_INVALID_ARG, "preconditioner belongs to another system");
    UFE_REQUIRE(opts->rtol > 0 && opts->maxit >= 0, UFE_ERR_INVALID_ARG, "bad solve options");
    UFE_REQUIRE(sys->ncomp == 1, UFE_ERR_UNSUPPORTED, "the coefficient gradient is defined for the Poisson problem");
    check_mem(mem);
    cudaStream_t s = sys->stream;
    const int64_t n = sys->mesh->n_dof, nc = sys->mesh->g.n_cells();
    DBuf<double> ub, jb, lb, gb;
    const double* ud = stage(ub, u, n, mem, s);
    const double* jd = stage(jb, dJdu, n, mem, s);
    double* ld = lambda;
    double* gd = dJdkappa;
    if (mem == UFE_MEM_HOST) {
      lb.alloc(n, s);
      copy_in(lb.p, lambda, n * 8, mem, s);
      ld = lb.p;
      gb.alloc(nc, s);
      gd = gb.p;
    }
    // A is symmetric positive definite, so the adjoint solve reuses the same BDDC-PCG
    pcg_solve(*B, jd, ld, *opts, info);
    kappa_gradient(*sys, ud, ld, gd, s);
    if (mem == UFE_MEM_HOST) {
      copy_out(lambda, ld, n * 8, mem, s);
      copy_out(dJdkappa, gd, nc * 8, mem, s);
    }
    UFE_CUDA(cudaStreamSynchronize(s));
  });
}

}  // extern "C"
