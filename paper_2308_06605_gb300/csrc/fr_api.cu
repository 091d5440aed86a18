// C ABI (include/fr.h): mesh lifetime, state transfer, residual and RK44 stages.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "fr_device.hpp"
#include "fr_part.hpp"

using namespace frx;

struct fr_mesh {
  HostMesh host;            // keeps xsol for fr_solution_points; bulk arrays released after upload
  fr_physics phys{};
  DevPhys dphys{};
  DevMesh dev{};
  cudaStream_t stream = nullptr;
  int device = 0;
  fr_status poisoned = FR_OK;
  std::string err;
  int64_t bytes = 0;
  double *h_scalar = nullptr;   // pinned host scalar for dt / flags
  // Source term arrays (allocated by fr_set_source).
  double *d_sigma = nullptr, *d_qref = nullptr;
  // 1D tables of a correction function c != 0 (device BasisT of the element arithmetic).
  void *d_vc = nullptr;
  // Eddy-viscosity closure (allocated by fr_set_closure).
  void *d_cw = nullptr;
  float *d_cscale = nullptr;
  // Domain decomposition (fr_mesh_create_part): halo lists and the device slot codes.
  bool is_part = false;
  HaloLists halo;
  int64_t *d_halo = nullptr;   // [n_halo] 2 I + side
  // Instrumentation: one event set per recorded residual evaluation.
  bool profiling = false;
  std::vector<PhaseEvents> ev_pool;
  size_t ev_used = 0;
};

static void clear_events(fr_mesh *m) {
  for (PhaseEvents &p : m->ev_pool)
    for (int k = 0; k < 4; ++k) {
      cudaEventDestroy(p.start[k]);
      cudaEventDestroy(p.stop[k]);
    }
  m->ev_pool.clear();
  m->ev_used = 0;
}

// Next event set when profiling, else null.
static const PhaseEvents *next_events(fr_mesh *m) {
  if (!m->profiling) return nullptr;
  if (m->ev_used == m->ev_pool.size()) {
    PhaseEvents p;
    for (int k = 0; k < 4; ++k) {
      if (cudaEventCreate(&p.start[k]) != cudaSuccess || cudaEventCreate(&p.stop[k]) != cudaSuccess) return nullptr;
    }
    m->ev_pool.push_back(p);
  }
  return &m->ev_pool[m->ev_used++];
}

static std::string g_create_error;
static std::mutex g_mutex;

static fr_status fail(fr_mesh *m, fr_status st, const std::string &msg) {
  if (m) {
    m->err = msg;
    if (st == FR_ECUDA || st == FR_ETIMEOUT) m->poisoned = st;
  } else {
    std::lock_guard<std::mutex> lk(g_mutex);
    g_create_error = msg;
  }
  return st;
}

static fr_status cuda_fail(fr_mesh *m, cudaError_t e, const char *what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(m, FR_ECUDA, msg);
}

#define FR_CUDA(m, call)                                 \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(m, e_, #call); \
  } while (0)

static fr_status check_mesh(fr_mesh *m) {
  if (!m) return FR_EINVAL;
  if (m->poisoned != FR_OK) return m->poisoned;
  return FR_OK;
}

// A part of a domain-decomposed mesh that shares interfaces with other parts needs their traces
// between the phases of a stage (fr_part_phase); whole-stage calls would read stale halo slots.
static fr_status refuse_halo(fr_mesh *m, const char *what) {
  if (m->is_part && !m->halo.iface.empty())
    return fail(m, FR_EUNSUPPORTED, std::string(what) + ": this part shares interfaces with other parts; use fr_part_phase");
  return FR_OK;
}

static void release(fr_mesh *m) {
  DevMesh &d = m->dev;
  double *dbl[] = {d.Q,  d.Un, d.acc, d.Rpart, d.metrics, d.liftfac, d.normals, d.Qtr,
                   d.Gtr, d.FI, d.h,   d.dtbuf, d.Qc,      d.Unc,     d.metrics_p, d.ptab};
  for (double *p : dbl)
    if (p) cudaFree(p);
  if (d.ef) cudaFree(d.ef);
  if (d.if_bc) cudaFree(d.if_bc);
  if (d.bcs) cudaFree(d.bcs);
  if (d.flag) cudaFree(d.flag);
  if (d.nu) cudaFree(d.nu);
  if (d.if_elem) cudaFree(d.if_elem);
  if (d.ef_p) cudaFree(d.ef_p);
  if (d.tri_slot) cudaFree(d.tri_slot);
  if (d.if_tri) cudaFree(d.if_tri);
  if (d.if_up) cudaFree(d.if_up);
  if (m->d_cw) cudaFree(m->d_cw);
  if (m->d_cscale) cudaFree(m->d_cscale);
  if (m->d_sigma) cudaFree(m->d_sigma);
  if (m->d_qref) cudaFree(m->d_qref);
  if (m->d_vc) cudaFree(m->d_vc);
  if (m->d_halo) cudaFree(m->d_halo);
  m->d_halo = nullptr;
  m->d_sigma = m->d_qref = nullptr;
  m->d_cw = nullptr;
  m->d_cscale = nullptr;
  if (m->h_scalar) cudaFreeHost(m->h_scalar);
  d = DevMesh{};
  m->h_scalar = nullptr;
}

template <typename T>
static fr_status dalloc(fr_mesh *m, T **p, size_t count) {
  size_t bytes = sizeof(T) * (count ? count : 1);
  cudaError_t e = cudaMalloc((void **)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(m, e == cudaErrorMemoryAllocation ? FR_ENOMEM : FR_ECUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  m->bytes += (int64_t)bytes;
  return FR_OK;
}

// Per-element orders (fr_mesh_desc.elem_p): NULL, or every entry in 1..7 and equal to p.
static fr_status check_elem_orders(const fr_mesh_desc *desc) {
  if (!desc->elem_p) return FR_OK;
  const int64_t n = desc->n_hex + desc->n_prism;
  for (int64_t e = 0; e < n; ++e)
    if (desc->elem_p[e] < 1 || desc->elem_p[e] > 7) {
      char buf[120];
      snprintf(buf, sizeof buf, "elem_p[%lld] = %d is outside 1..7", (long long)e, (int)desc->elem_p[e]);
      return fail(nullptr, FR_EINVAL, buf);
    }
  for (int64_t e = 0; e < n; ++e)
    if (desc->elem_p[e] != desc->p) {
      char buf[200];
      snprintf(buf, sizeof buf,
               "elem_p[%lld] = %d differs from p = %d: meshes of mixed orders (p-nonconforming interfaces) are "
               "not built",
               (long long)e, (int)desc->elem_p[e], (int)desc->p);
      return fail(nullptr, FR_EUNSUPPORTED, buf);
    }
  return FR_OK;
}

// Checks of a mesh description and physics before anything is allocated.
static fr_status validate_create(const fr_mesh_desc *desc, const fr_physics *phys) {
  if (!desc || !phys) return fail(nullptr, FR_EINVAL, "desc or phys is NULL");
  if (desc->p < 1 || desc->p > 7) return fail(nullptr, FR_EINVAL, "p must be in 1..7");
  if (desc->n_hex < 0 || desc->n_prism < 0 || desc->n_hex + desc->n_prism <= 0 || (desc->n_hex > 0 && !desc->hex) ||
      (desc->n_prism > 0 && !desc->prism) || desc->n_nodes <= 0 || !desc->xyz)
    return fail(nullptr, FR_EINVAL, "empty mesh or NULL arrays");
  if (desc->n_bface < 0 || (desc->n_bface > 0 && (!desc->bface_nodes || !desc->bface_tag)))
    return fail(nullptr, FR_EINVAL, "bad boundary-face arrays");
  if (desc->n_bc < 0 || (desc->n_bc > 0 && !desc->bc) || desc->n_periodic < 0 ||
      (desc->n_periodic > 0 && !desc->periodic))
    return fail(nullptr, FR_EINVAL, "bad boundary-condition or periodic arrays");
  if (fr_status so = check_elem_orders(desc); so != FR_OK) return so;
  if (!(phys->gamma > 1.0) || !(phys->R > 0.0) || !(phys->mu >= 0.0) || !(phys->Pr > 0.0) ||
      !(phys->br2_eta >= 0.0))
    return fail(nullptr, FR_EINVAL, "bad physical parameters");
  if (phys->inviscid != FR_RUSANOV && phys->inviscid != FR_ROE)
    return fail(nullptr, FR_EINVAL, "unknown inviscid flux");
  if (phys->viscous != FR_VISC_NONE && phys->viscous != FR_VISC_BR2 && phys->viscous != FR_VISC_LDG)
    return fail(nullptr, FR_EINVAL, "unknown viscous scheme");
  if (phys->viscous == FR_VISC_LDG && !(phys->ldg_tau >= 0.0))
    return fail(nullptr, FR_EINVAL, "LDG penalty must be non-negative");
  if (phys->precision != FR_PREC_FP64 && phys->precision != FR_PREC_MIXED && phys->precision != FR_PREC_MIXED_TC &&
      phys->precision != FR_PREC_MIXED_VF32)
    return fail(nullptr, FR_EINVAL, "unknown precision");
  if (phys->precision == FR_PREC_MIXED_VF32 && phys->vcjh_c != 0.0)
    return fail(nullptr, FR_EUNSUPPORTED, "FR_PREC_MIXED_VF32 is built for the DG-equivalent correction (c = 0)");
  if (!vcjh_in_family(desc->p, phys->vcjh_c))
    return fail(nullptr, FR_EINVAL, "correction parameter c outside the energy-stable family (1 + eta <= 0)");
  if (phys->vcjh_c != 0.0 && desc->n_prism > 0)
    return fail(nullptr, FR_EUNSUPPORTED, "correction functions with c != 0 are built for hexahedral meshes only");
  for (int k = 0; k < desc->n_bc; ++k) {
    const fr_bc &b = desc->bc[k];
    if (b.kind < FR_BC_WALL_ISOTHERMAL || b.kind > FR_BC_DIRICHLET)
      return fail(nullptr, FR_EINVAL, "unknown boundary-condition kind");
    if (b.kind == FR_BC_WALL_ISOTHERMAL && !(b.params[0] > 0.0))
      return fail(nullptr, FR_EINVAL, "wall temperature must be positive");
    if (b.kind == FR_BC_CHAR_OUTFLOW && !(b.params[0] > 0.0))
      return fail(nullptr, FR_EINVAL, "outflow pressure must be positive");
    if (b.kind == FR_BC_CHAR_INFLOW &&
        (!(b.params[0] > 0.0) || !(b.params[1] > 0.0) ||
         !(b.params[2] * b.params[2] + b.params[3] * b.params[3] + b.params[4] * b.params[4] > 0.0)))
      return fail(nullptr, FR_EINVAL, "inflow needs positive total pressure/temperature and a direction");
    if (b.kind == FR_BC_DIRICHLET && !(b.params[0] > 0.0))
      return fail(nullptr, FR_EINVAL, "Dirichlet density must be positive");
  }

  return FR_OK;
}

static fr_status finish_create(fr_mesh *m, const fr_physics *phys, uintptr_t stream, fr_mesh **out);

extern "C" fr_status fr_mesh_create(const fr_mesh_desc *desc, const fr_physics *phys, uintptr_t stream,
                                    fr_mesh **out) {
  if (!out) return fail(nullptr, FR_EINVAL, "out is NULL");
  *out = nullptr;
  if (fr_status sv = validate_create(desc, phys); sv != FR_OK) return sv;
  fr_mesh *m = new (std::nothrow) fr_mesh();
  if (!m) return fail(nullptr, FR_ENOMEM, "host allocation failed");
  std::string err;
  fr_status st;
  try {
    st = build_host_mesh(desc, m->host, err, phys->vcjh_c);
  } catch (const std::bad_alloc &) {
    st = FR_ENOMEM;
    err = "host allocation failed while building the mesh";
  }
  if (st != FR_OK) {
    delete m;
    return fail(nullptr, st, err);
  }
  return finish_create(m, phys, stream, out);
}

// Device set-up of a mesh whose host part (m->host) is built: physics constants, buffers,
// uploads.  Takes ownership of m (freed on failure).
static fr_status finish_create(fr_mesh *m, const fr_physics *phys, uintptr_t stream, fr_mesh **out) {
  fr_status st = FR_OK;
  m->phys = *phys;
  m->stream = (cudaStream_t)stream;
  DevPhys &dp = m->dphys;
  dp.gamma = phys->gamma;
  dp.R = phys->R;
  dp.mu = phys->mu;
  dp.kappa = phys->mu * phys->gamma * phys->R / ((phys->gamma - 1.0) * phys->Pr);
  dp.viscous = (phys->viscous != FR_VISC_NONE && phys->mu > 0.0) ? 1 : 0;
  dp.ldg = phys->viscous == FR_VISC_LDG ? 1 : 0;
  dp.ldg_tau = dp.ldg ? phys->ldg_tau : 0.0;
  dp.eta = dp.ldg ? 0.0 : phys->br2_eta;     // LDG's face gradients carry no lifting term
  dp.inviscid = phys->inviscid;
  {
    const double vals[11] = {dp.gamma, dp.gamma - 1.0, (dp.gamma - 1.0) / dp.R, dp.mu, -2.0 * dp.mu / 3.0,
                             dp.kappa, dp.eta, 0.0, 0.5, 1.0, dp.ldg_tau};
    double *dd[11] = {&dp.d.gamma, &dp.d.gm1, &dp.d.cT, &dp.d.mu, &dp.d.m2mu3, &dp.d.kappa, &dp.d.eta,
                      &dp.d.zero, &dp.d.half, &dp.d.one, &dp.d.tau};
    df32 *ff[11] = {&dp.f.gamma, &dp.f.gm1, &dp.f.cT, &dp.f.mu, &dp.f.m2mu3, &dp.f.kappa, &dp.f.eta,
                    &dp.f.zero, &dp.f.half, &dp.f.one, &dp.f.tau};
    float *sf[11] = {&dp.s.gamma, &dp.s.gm1, &dp.s.cT, &dp.s.mu, &dp.s.m2mu3, &dp.s.kappa, &dp.s.eta,
                     &dp.s.zero, &dp.s.half, &dp.s.one, &dp.s.tau};
    for (int k = 0; k < 11; ++k) {
      *dd[k] = vals[k];
      *ff[k] = df_split_host(vals[k]);
      *sf[k] = (float)vals[k];
    }
  }

  auto bail = [&](fr_status s) {
    std::string msg = m->err;
    release(m);
    delete m;
    return fail(nullptr, s, msg);
  };
  cudaError_t ce = cudaGetDevice(&m->device);
  if (ce != cudaSuccess) { m->err = cudaGetErrorString(ce); return bail(FR_ECUDA); }
  {
    static bool uploaded[64] = {false};
    std::lock_guard<std::mutex> lk(g_mutex);
    if (m->device < 64 && !uploaded[m->device]) {
      ce = upload_basis_tables();
      if (ce != cudaSuccess) { m->err = std::string("basis upload: ") + cudaGetErrorString(ce); }
      else uploaded[m->device] = true;
    }
  }
  if (ce != cudaSuccess) return bail(FR_ECUDA);
  HostMesh &h = m->host;
  DevMesh &d = m->dev;
  d.p = h.p; d.N = h.N; d.Np = h.Np; d.Nf = h.Nf;
  d.E = h.E; d.n_if = h.n_if; d.n_interior = h.n_interior;
  d.Ep = h.Ep; d.Nt = h.Nt; d.Npp = h.Npp;
  d.mixed = (phys->precision == FR_PREC_MIXED || phys->precision == FR_PREC_MIXED_TC ||
             phys->precision == FR_PREC_MIXED_VF32) ? 1 : 0;
  d.tc = (phys->precision == FR_PREC_MIXED_TC) ? 1 : 0;
  d.vf32 = (phys->precision == FR_PREC_MIXED_VF32) ? 1 : 0;
  const size_t nsol = ((size_t)h.E * h.Np + (size_t)h.Ep * h.Npp) * 5;
  const size_t G = (size_t)(h.E + h.Ep);
  const size_t Nf = h.Nf;
  if ((st = dalloc(m, &d.Q, nsol)) || (st = dalloc(m, &d.Un, nsol)) || (st = dalloc(m, &d.acc, nsol)) ||
      (st = dalloc(m, &d.Rpart, nsol)) || (st = dalloc(m, &d.metrics, h.metrics.size())) ||
      (st = dalloc(m, &d.liftfac, h.liftfac.size())) || (st = dalloc(m, &d.normals, h.normals.size())) ||
      (st = dalloc(m, &d.Qtr, (size_t)h.n_if * 2 * 5 * Nf)) ||
      (st = dalloc(m, &d.Gtr, (size_t)h.n_if * 2 * 15 * Nf)) || (st = dalloc(m, &d.FI, (size_t)h.n_if * 5 * Nf)) ||
      (st = dalloc(m, &d.h, G)) || (st = dalloc(m, &d.dtbuf, G + 1)) ||
      (st = dalloc(m, &d.ef, h.ef.size())) || (st = dalloc(m, &d.if_bc, h.if_bc.size())) ||
      (st = dalloc(m, &d.bcs, h.bcs.size())) || (st = dalloc(m, &d.flag, 1)) ||
      (d.mixed && ((st = dalloc(m, &d.Qc, nsol)) || (st = dalloc(m, &d.Unc, nsol)))))
    return bail(st);
  if (h.Ep > 0 && ((st = dalloc(m, &d.ef_p, h.ef_p.size())) || (st = dalloc(m, &d.metrics_p, h.metrics_p.size())) ||
                   (st = dalloc(m, &d.ptab, h.ptab.size())) || (st = dalloc(m, &d.tri_slot, h.tri_slot.size())) ||
                   (st = dalloc(m, &d.if_tri, h.if_tri.size()))))
    return bail(st);
  if ((st = dalloc(m, &d.if_up, h.if_up.size()))) return bail(st);
  if (phys->vcjh_c != 0.0) {
    ce = vcjh_basis_create(h.p, phys->vcjh_c, d.mixed, &m->d_vc);
    if (ce != cudaSuccess) {
      m->err = std::string("correction tables: ") + cudaGetErrorString(ce);
      return bail(ce == cudaErrorMemoryAllocation ? FR_ENOMEM : FR_ECUDA);
    }
    dp.vc_basis = m->d_vc;
  }
  if (d.mixed) {
    // Geometry in the element arithmetic's format: each double becomes a df32 (hi, lo) pair
    // stored in the same 8-byte slot.
    for (std::vector<double> *v : {&h.metrics, &h.liftfac, &h.normals, &h.metrics_p, &h.ptab})
      for (double &x : *v) {
        df32 p = df_split_host(x);
        std::memcpy(&x, &p, sizeof(double));
      }
  }
  ce = cudaMallocHost((void **)&m->h_scalar, 4 * sizeof(double));
  if (ce != cudaSuccess) { m->err = cudaGetErrorString(ce); return bail(FR_ENOMEM); }
  struct Up { void *dst; const void *src; size_t bytes; } ups[] = {
      {d.metrics, h.metrics.data(), h.metrics.size() * sizeof(double)},
      {d.liftfac, h.liftfac.data(), h.liftfac.size() * sizeof(double)},
      {d.normals, h.normals.data(), h.normals.size() * sizeof(double)},
      {d.h, h.h.data(), h.h.size() * sizeof(double)},
      {d.ef, h.ef.data(), h.ef.size() * sizeof(int32_t)},
      {d.if_bc, h.if_bc.data(), h.if_bc.size() * sizeof(int32_t)},
      {d.bcs, h.bcs.data(), h.bcs.size() * sizeof(fr_bc)},
      {d.ef_p, h.ef_p.data(), h.ef_p.size() * sizeof(int32_t)},
      {d.metrics_p, h.metrics_p.data(), h.metrics_p.size() * sizeof(double)},
      {d.ptab, h.ptab.data(), h.ptab.size() * sizeof(double)},
      {d.tri_slot, h.tri_slot.data(), h.tri_slot.size() * sizeof(int32_t)},
      {d.if_tri, h.if_tri.data(), h.if_tri.size() * sizeof(int8_t)},
      {d.if_up, h.if_up.data(), h.if_up.size() * sizeof(int8_t)},
  };
  for (const Up &u : ups) {
    if (u.bytes == 0) continue;
    ce = cudaMemcpyAsync(u.dst, u.src, u.bytes, cudaMemcpyHostToDevice, m->stream);
    if (ce != cudaSuccess) { m->err = std::string("upload: ") + cudaGetErrorString(ce); return bail(FR_ECUDA); }
  }
  // Interface buffers start at zero; the state is undefined until fr_set_state.
  ce = cudaMemsetAsync(d.Qtr, 0, (size_t)h.n_if * 2 * 5 * Nf * sizeof(double), m->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(d.Gtr, 0, (size_t)h.n_if * 2 * 15 * Nf * sizeof(double), m->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(d.flag, 0, sizeof(int), m->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(m->stream);
  if (ce != cudaSuccess) { m->err = std::string("init: ") + cudaGetErrorString(ce); return bail(FR_ECUDA); }
  // Bulk host copies are no longer needed.
  std::vector<double>().swap(h.metrics);
  std::vector<double>().swap(h.liftfac);
  std::vector<double>().swap(h.normals);
  std::vector<double>().swap(h.metrics_p);
  *out = m;
  return FR_OK;
}

extern "C" fr_status fr_mesh_query(const fr_mesh *m, fr_mesh_info *info) {
  if (!m || !info) return FR_EINVAL;
  info->n_elem = m->host.E;
  info->p = m->host.p;
  info->n_pts = m->host.Np;
  info->n_iface = m->host.n_interior;
  info->n_bface = m->host.n_if - m->host.n_interior;
  info->device_bytes = m->bytes;
  info->n_prism = m->host.Ep;
  info->n_pts_prism = m->host.Npp;
  info->n_points = m->host.E * m->host.Np + m->host.Ep * m->host.Npp;
  info->device = m->device;
  return FR_OK;
}

extern "C" fr_status fr_mesh_inspect(const fr_mesh_desc *desc, fr_mesh_info *info, double *xyz_host,
                                     double *metrics_host, int32_t *ef_host, double *normals_host,
                                     int32_t *ef_prism_host, int32_t *tri_slot_host) {
  if (!desc || !info) return fail(nullptr, FR_EINVAL, "desc or info is NULL");
  if (desc->p < 1 || desc->p > 7) return fail(nullptr, FR_EINVAL, "p must be in 1..7");
  if (desc->n_hex < 0 || desc->n_prism < 0 || desc->n_hex + desc->n_prism <= 0 || (desc->n_hex > 0 && !desc->hex) ||
      (desc->n_prism > 0 && !desc->prism) || desc->n_nodes <= 0 || !desc->xyz)
    return fail(nullptr, FR_EINVAL, "empty mesh or NULL arrays");
  if (desc->n_bface < 0 || (desc->n_bface > 0 && (!desc->bface_nodes || !desc->bface_tag)))
    return fail(nullptr, FR_EINVAL, "bad boundary-face arrays");
  if (desc->n_bc < 0 || (desc->n_bc > 0 && !desc->bc) || desc->n_periodic < 0 ||
      (desc->n_periodic > 0 && !desc->periodic))
    return fail(nullptr, FR_EINVAL, "bad boundary-condition or periodic arrays");
  if (fr_status so = check_elem_orders(desc); so != FR_OK) return so;
  HostMesh h;
  std::string err;
  fr_status st;
  try {
    st = build_host_mesh(desc, h, err);
  } catch (const std::bad_alloc &) {
    st = FR_ENOMEM;
    err = "host allocation failed while building the mesh";
  }
  if (st != FR_OK) return fail(nullptr, st, err);
  info->n_elem = h.E;
  info->p = h.p;
  info->n_pts = h.Np;
  info->n_iface = h.n_interior;
  info->n_bface = h.n_if - h.n_interior;
  info->device_bytes = 0;
  info->n_prism = h.Ep;
  info->n_pts_prism = h.Npp;
  info->n_points = h.E * h.Np + h.Ep * h.Npp;
  info->device = -1;
  if (xyz_host) std::memcpy(xyz_host, h.xsol.data(), h.xsol.size() * sizeof(double));
  if (metrics_host) {
    std::memcpy(metrics_host, h.metrics.data(), h.metrics.size() * sizeof(double));
    std::memcpy(metrics_host + h.metrics.size(), h.metrics_p.data(), h.metrics_p.size() * sizeof(double));
  }
  if (ef_host) std::memcpy(ef_host, h.ef.data(), h.ef.size() * sizeof(int32_t));
  if (normals_host) std::memcpy(normals_host, h.normals.data(), h.normals.size() * sizeof(double));
  if (ef_prism_host) std::memcpy(ef_prism_host, h.ef_p.data(), h.ef_p.size() * sizeof(int32_t));
  if (tri_slot_host && !h.tri_slot.empty())
    std::memcpy(tri_slot_host, h.tri_slot.data(), h.tri_slot.size() * sizeof(int32_t));
  return FR_OK;
}

extern "C" fr_status fr_solution_points(fr_mesh *m, double *xyz) {
  fr_status st = check_mesh(m);
  if (st) return st;
  if (!xyz) return fail(m, FR_EINVAL, "xyz is NULL");
  std::memcpy(xyz, m->host.xsol.data(), m->host.xsol.size() * sizeof(double));
  return FR_OK;
}

// Bytes of a state or residual in the canonical layout (hexahedral points, then prism points).
static size_t state_bytes(const DevMesh &d) {
  return ((size_t)d.E * d.Np + (size_t)d.Ep * d.Npp) * 5 * sizeof(double);
}

static cudaMemcpyKind kind_of(int where, bool to_device) {
  if (where == FR_DEVICE) return cudaMemcpyDeviceToDevice;
  return to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
}

extern "C" fr_status fr_set_state(fr_mesh *m, const double *Q, int32_t where) {
  fr_status st = check_mesh(m);
  if (st) return st;
  if (!Q || (where != FR_HOST && where != FR_DEVICE)) return fail(m, FR_EINVAL, "bad state pointer or where");
  const size_t bytes = state_bytes(m->dev);
  FR_CUDA(m, cudaMemcpyAsync(m->dev.Q, Q, bytes, kind_of(where, true), m->stream));
  FR_CUDA(m, cudaMemcpyAsync(m->dev.Un, m->dev.Q, bytes, cudaMemcpyDeviceToDevice, m->stream));
  FR_CUDA(m, launch_state_copy(m->dev, m->stream));
  if (where == FR_HOST) FR_CUDA(m, cudaStreamSynchronize(m->stream));
  return FR_OK;
}

extern "C" fr_status fr_get_state(fr_mesh *m, double *Q, int32_t where) {
  fr_status st = check_mesh(m);
  if (st) return st;
  if (!Q || (where != FR_HOST && where != FR_DEVICE)) return fail(m, FR_EINVAL, "bad state pointer or where");
  const size_t bytes = state_bytes(m->dev);
  FR_CUDA(m, cudaMemcpyAsync(Q, m->dev.Q, bytes, kind_of(where, false), m->stream));
  if (where == FR_HOST) FR_CUDA(m, cudaStreamSynchronize(m->stream));
  return FR_OK;
}

extern "C" fr_status fr_residual(fr_mesh *m, double t, double *R, int32_t where) {
  (void)t;
  fr_status st = check_mesh(m);
  if (st) return st;
  if ((st = refuse_halo(m, "fr_residual"))) return st;
  if (!R || (where != FR_HOST && where != FR_DEVICE)) return fail(m, FR_EINVAL, "bad residual pointer or where");
  double *dst = (where == FR_DEVICE) ? R : m->dev.acc;   // acc is free outside an RK step
  FR_CUDA(m, launch_residual(m->dev, m->dphys, MODE_RESIDUAL, 0, 0.0, dst, m->stream, next_events(m)));
  if (where == FR_HOST) {
    const size_t bytes = state_bytes(m->dev);
    FR_CUDA(m, cudaMemcpyAsync(R, dst, bytes, cudaMemcpyDeviceToHost, m->stream));
    FR_CUDA(m, cudaStreamSynchronize(m->stream));
  }
  return FR_OK;
}

extern "C" fr_status fr_rk_stage(fr_mesh *m, int32_t scheme, int32_t stage, double t, double dt) {
  (void)t;
  fr_status st = check_mesh(m);
  if (st) return st;
  if ((st = refuse_halo(m, "fr_rk_stage"))) return st;
  int mode, last;
  switch (scheme) {
    case FR_RK44: mode = MODE_RK; last = 3; break;
    case FR_SSPRK33: mode = MODE_SSP33; last = 2; break;
    case FR_SSPRK104: mode = MODE_SSP104; last = 9; break;
    default: return fail(m, FR_EINVAL, "unknown Runge-Kutta scheme");
  }
  if (stage < 0 || stage > last || !std::isfinite(dt)) return fail(m, FR_EINVAL, "bad stage or dt");
  FR_CUDA(m, launch_residual(m->dev, m->dphys, mode, stage, dt, nullptr, m->stream, next_events(m)));
  if (stage == last) {
    int *hflag = reinterpret_cast<int *>(m->h_scalar);
    FR_CUDA(m, cudaMemcpyAsync(hflag, m->dev.flag, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    FR_CUDA(m, cudaStreamSynchronize(m->stream));
    if (*hflag) {
      const int f = *hflag;
      FR_CUDA(m, cudaMemsetAsync(m->dev.flag, 0, sizeof(int), m->stream));
      if (f & 2) return fail(m, FR_ETIMEOUT, "a tensor-core kernel gave up waiting for its copies or MMAs");
      return fail(m, FR_ENONFINITE, "non-finite value in the updated state");
    }
  }
  return FR_OK;
}

extern "C" fr_status fr_max_dt(fr_mesh *m, double cfl, double *dt) {
  fr_status st = check_mesh(m);
  if (st) return st;
  if (!dt || !(cfl > 0.0)) return fail(m, FR_EINVAL, "bad dt pointer or cfl");
  double *d_out = m->dev.dtbuf + m->dev.E + m->dev.Ep;
  FR_CUDA(m, launch_max_dt(m->dev, m->dphys, cfl, d_out, m->stream));
  FR_CUDA(m, cudaMemcpyAsync(m->h_scalar, d_out, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  FR_CUDA(m, cudaStreamSynchronize(m->stream));
  *dt = m->h_scalar[0];
  return FR_OK;
}

// float -> bfloat16 bits, round to nearest even (NaN kept quiet).
static uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

extern "C" fr_status fr_set_closure(fr_mesh *m, const float *params, const float *scales, int32_t enable) {
  fr_status st = check_mesh(m);
  if (st) return st;
  if (m->is_part)
    return fail(m, FR_EUNSUPPORTED, "fr_set_closure: the closure needs the eddy viscosity of remote elements; not built for parts");
  if (!enable) {
    m->dphys.closure = 0;
    return FR_OK;
  }
  if (!params || !scales) return fail(m, FR_EINVAL, "closure parameters or scales are NULL");
  if (!m->dphys.viscous) return fail(m, FR_EINVAL, "the closure needs the viscous (BR2) path");
  if (m->dev.Ep > 0) return fail(m, FR_EUNSUPPORTED, "the closure is built for hexahedral meshes only");
  for (int k = 0; k < 11; ++k)
    if (!(scales[11 + k] > 0.f)) return fail(m, FR_EINVAL, "closure input scales must be positive");
  const int n = FR_CLOSURE_NPARAMS;
  std::vector<uint16_t> w(n);
  for (int k = 0; k < n; ++k) w[k] = bf16_bits(params[k]);
  DevMesh &d = m->dev;
  if (!m->d_cw) {
    fr_status s;
    if ((s = dalloc(m, reinterpret_cast<uint16_t **>(&m->d_cw), (size_t)n)) || (s = dalloc(m, &m->d_cscale, 23)) ||
        (s = dalloc(m, &d.nu, (size_t)d.E)) || (s = dalloc(m, &d.if_elem, m->host.if_elem.size())))
      return s;
    FR_CUDA(m, cudaMemcpyAsync(d.if_elem, m->host.if_elem.data(), m->host.if_elem.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, m->stream));
    FR_CUDA(m, cudaMemsetAsync(d.nu, 0, sizeof(float) * d.E, m->stream));
  }
  FR_CUDA(m, cudaMemcpyAsync(m->d_cw, w.data(), sizeof(uint16_t) * n, cudaMemcpyHostToDevice, m->stream));
  FR_CUDA(m, cudaMemcpyAsync(m->d_cscale, scales, sizeof(float) * 23, cudaMemcpyHostToDevice, m->stream));
  FR_CUDA(m, cudaStreamSynchronize(m->stream));
  m->dphys.closure = 1;
  m->dphys.cw = m->d_cw;
  m->dphys.cscale = m->d_cscale;
  m->dphys.cp_prt = m->phys.gamma * m->phys.R / (m->phys.gamma - 1.0) / FR_CLOSURE_PRT;
  return FR_OK;
}

extern "C" fr_status fr_set_source(fr_mesh *m, const double *accel, const double *sigma, const double *Q_ref) {
  fr_status st = check_mesh(m);
  if (st) return st;
  if ((sigma == nullptr) != (Q_ref == nullptr)) return fail(m, FR_EINVAL, "sigma and Q_ref go together");
  DevPhys &dp = m->dphys;
  dp.src_body = accel ? 1 : 0;
  for (int c = 0; c < 3; ++c) dp.accel[c] = accel ? accel[c] : 0.0;
  if (accel)
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(accel[c])) return fail(m, FR_EINVAL, "non-finite body acceleration");
  dp.src_sponge = 0;
  if (!sigma) return FR_OK;
  const size_t n = (size_t)m->dev.E * m->dev.Np + (size_t)m->dev.Ep * m->dev.Npp;
  for (size_t i = 0; i < n; ++i)
    if (!(sigma[i] >= 0.0) || !std::isfinite(sigma[i])) return fail(m, FR_EINVAL, "sponge strength must be >= 0");
  if (!m->d_sigma) {
    fr_status s;
    if ((s = dalloc(m, &m->d_sigma, n)) || (s = dalloc(m, &m->d_qref, n * 5))) return s;
  }
  FR_CUDA(m, cudaMemcpyAsync(m->d_sigma, sigma, n * sizeof(double), cudaMemcpyHostToDevice, m->stream));
  FR_CUDA(m, cudaMemcpyAsync(m->d_qref, Q_ref, n * 5 * sizeof(double), cudaMemcpyHostToDevice, m->stream));
  FR_CUDA(m, cudaStreamSynchronize(m->stream));
  dp.sigma = m->d_sigma;
  dp.Q_ref = m->d_qref;
  dp.src_sponge = 1;
  return FR_OK;
}

extern "C" fr_status fr_closure_nu(fr_mesh *m, float *nu_host) {
  fr_status st = check_mesh(m);
  if (st) return st;
  if (!nu_host) return fail(m, FR_EINVAL, "nu is NULL");
  if (!m->dev.nu) return fail(m, FR_EINVAL, "no closure set");
  FR_CUDA(m, cudaMemcpyAsync(nu_host, m->dev.nu, sizeof(float) * m->dev.E, cudaMemcpyDeviceToHost, m->stream));
  FR_CUDA(m, cudaStreamSynchronize(m->stream));
  return FR_OK;
}

extern "C" fr_status fr_profile(fr_mesh *m, int32_t enable) {
  fr_status st = check_mesh(m);
  if (st) return st;
  FR_CUDA(m, cudaStreamSynchronize(m->stream));
  clear_events(m);
  m->profiling = enable != 0;
  return FR_OK;
}

extern "C" fr_status fr_profile_read(fr_mesh *m, double *ms, int64_t *launches, int32_t n) {
  fr_status st = check_mesh(m);
  if (st) return st;
  if (!ms || !launches || n < 0) return fail(m, FR_EINVAL, "bad profile buffers");
  FR_CUDA(m, cudaStreamSynchronize(m->stream));
  for (int k = 0; k < n; ++k) { ms[k] = 0.0; launches[k] = 0; }
  for (size_t i = 0; i < m->ev_used; ++i)
    for (int k = 0; k < 4 && k < n; ++k) {
      float t = 0.f;
      FR_CUDA(m, cudaEventElapsedTime(&t, m->ev_pool[i].start[k], m->ev_pool[i].stop[k]));
      ms[k] += t;
      launches[k] += 1;
    }
  return FR_OK;
}

extern "C" void fr_free(fr_mesh *m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  clear_events(m);
  release(m);
  delete m;
}

// ------------------------------------------------------------------ domain decomposition

// Element centroids (mean of the corner vertices) and work weights (solution points).
static void element_centroids(const fr_mesh_desc *d, std::vector<double> &cent, std::vector<double> &w) {
  const int hn = d->hex_nodes == 0 ? 8 : d->hex_nodes, pn = d->prism_nodes == 0 ? 6 : d->prism_nodes;
  const int N = d->p + 1;
  const int64_t n = d->n_hex + d->n_prism;
  cent.assign((size_t)n * 3, 0.0);
  w.assign((size_t)n, 0.0);
  for (int64_t e = 0; e < n; ++e) {
    const bool hex = e < d->n_hex;
    const int64_t *v = hex ? d->hex + e * hn : d->prism + (e - d->n_hex) * pn;
    const int nc = hex ? 8 : 6;
    for (int k = 0; k < nc; ++k)
      for (int c = 0; c < 3; ++c) cent[e * 3 + c] += d->xyz[v[k] * 3 + c] / nc;
    w[e] = hex ? (double)N * N * N : (double)N * N * (N + 1) / 2;
  }
}

static fr_status check_vertex_ids(const fr_mesh_desc *d) {
  const int hn = d->hex_nodes == 0 ? 8 : d->hex_nodes, pn = d->prism_nodes == 0 ? 6 : d->prism_nodes;
  for (int64_t i = 0; i < d->n_hex * hn; ++i)
    if (d->hex[i] < 0 || d->hex[i] >= d->n_nodes) return fail(nullptr, FR_EMESH, "vertex id out of range");
  for (int64_t i = 0; i < d->n_prism * pn; ++i)
    if (d->prism[i] < 0 || d->prism[i] >= d->n_nodes) return fail(nullptr, FR_EMESH, "vertex id out of range");
  return FR_OK;
}

static fr_status check_desc_arrays(const fr_mesh_desc *desc) {
  if (desc->p < 1 || desc->p > 7) return fail(nullptr, FR_EINVAL, "p must be in 1..7");
  if (desc->n_hex < 0 || desc->n_prism < 0 || desc->n_hex + desc->n_prism <= 0 || (desc->n_hex > 0 && !desc->hex) ||
      (desc->n_prism > 0 && !desc->prism) || desc->n_nodes <= 0 || !desc->xyz)
    return fail(nullptr, FR_EINVAL, "empty mesh or NULL arrays");
  if (desc->n_bface < 0 || (desc->n_bface > 0 && (!desc->bface_nodes || !desc->bface_tag)))
    return fail(nullptr, FR_EINVAL, "bad boundary-face arrays");
  if (desc->n_bc < 0 || (desc->n_bc > 0 && !desc->bc) || desc->n_periodic < 0 ||
      (desc->n_periodic > 0 && !desc->periodic))
    return fail(nullptr, FR_EINVAL, "bad boundary-condition or periodic arrays");
  return FR_OK;
}

// Partition with element weights: the solution-point count of each element, or, when the costs
// per solution point of a hexahedron and of a prism are given (> 0), that count times the cost.
static fr_status partition_weighted(const fr_mesh_desc *desc, int32_t n_parts, double cost_hex, double cost_prism,
                                    int32_t *part) {
  if (!desc || !part) return fail(nullptr, FR_EINVAL, "desc or part is NULL");
  if (!(cost_hex > 0.0) || !(cost_prism > 0.0) || !std::isfinite(cost_hex) || !std::isfinite(cost_prism))
    return fail(nullptr, FR_EINVAL, "costs per solution point must be finite and positive");
  if (fr_status sv = check_desc_arrays(desc); sv != FR_OK) return sv;
  if (fr_status sv = check_vertex_ids(desc); sv != FR_OK) return sv;
  std::vector<double> cent, w;
  std::vector<int32_t> pv;
  std::string err;
  element_centroids(desc, cent, w);
  for (int64_t e = 0; e < (int64_t)w.size(); ++e) w[e] *= e < desc->n_hex ? cost_hex : cost_prism;
  fr_status st = partition_elements(cent, w, n_parts, pv, err);
  if (st != FR_OK) return fail(nullptr, st, err);
  std::memcpy(part, pv.data(), pv.size() * sizeof(int32_t));
  return FR_OK;
}

extern "C" fr_status fr_partition(const fr_mesh_desc *desc, int32_t n_parts, int32_t *part) {
  return partition_weighted(desc, n_parts, 1.0, 1.0, part);
}

extern "C" fr_status fr_partition_cost(const fr_mesh_desc *desc, int32_t n_parts, double cost_hex, double cost_prism,
                                       int32_t *part) {
  return partition_weighted(desc, n_parts, cost_hex, cost_prism, part);
}

// Host build of part `rank`: the global connectivity, then the part and its halo lists.
static fr_status build_part(const fr_mesh_desc *desc, const int32_t *part, int32_t rank, HostMesh &local,
                            HaloLists &halo) {
  if (!part || rank < 0) return fail(nullptr, FR_EINVAL, "part is NULL or rank negative");
  const int64_t n = desc->n_hex + desc->n_prism;
  for (int64_t e = 0; e < n; ++e)
    if (part[e] < 0) return fail(nullptr, FR_EINVAL, "negative part id");
  HostMesh g;
  std::string err;
  fr_status st;
  try {
    st = build_host_mesh(desc, g, err, 0.0);
    if (st == FR_OK) st = extract_part(g, std::vector<int32_t>(part, part + n), rank, local, halo, err);
  } catch (const std::bad_alloc &) {
    st = FR_ENOMEM;
    err = "host allocation failed while building the part";
  }
  return st == FR_OK ? FR_OK : fail(nullptr, st, err);
}

static void fill_part_info(const HostMesh &h, const HaloLists &halo, fr_part_info *info) {
  info->n_elem = h.E + h.Ep;
  info->n_iface = h.n_interior;
  info->n_bface = h.n_if - h.n_interior;
  info->n_peers = (int32_t)halo.peers.size();
  info->n_halo = (int64_t)halo.iface.size();
}

static void copy_halo(const HaloLists &halo, int32_t *peers, int64_t *peer_begin, int64_t *gid, int64_t *elem_global) {
  if (peers && !halo.peers.empty()) std::memcpy(peers, halo.peers.data(), halo.peers.size() * sizeof(int32_t));
  if (peer_begin) std::memcpy(peer_begin, halo.peer_begin.data(), halo.peer_begin.size() * sizeof(int64_t));
  if (gid && !halo.gid.empty()) std::memcpy(gid, halo.gid.data(), halo.gid.size() * sizeof(int64_t));
  if (elem_global) std::memcpy(elem_global, halo.elem_global.data(), halo.elem_global.size() * sizeof(int64_t));
}

extern "C" fr_status fr_part_inspect(const fr_mesh_desc *desc, const int32_t *part, int32_t rank, fr_part_info *info,
                                     int32_t *peers, int64_t *peer_begin, int64_t *gid, int64_t *elem_global) {
  if (!desc || !info) return fail(nullptr, FR_EINVAL, "desc or info is NULL");
  if (fr_status sv = check_desc_arrays(desc); sv != FR_OK) return sv;
  HostMesh h;
  HaloLists halo;
  if (fr_status st = build_part(desc, part, rank, h, halo); st != FR_OK) return st;
  fill_part_info(h, halo, info);
  copy_halo(halo, peers, peer_begin, gid, elem_global);
  return FR_OK;
}

extern "C" fr_status fr_mesh_create_part(const fr_mesh_desc *desc, const fr_physics *phys, const int32_t *part,
                                         int32_t rank, uintptr_t stream, fr_mesh **out) {
  if (!out) return fail(nullptr, FR_EINVAL, "out is NULL");
  *out = nullptr;
  if (fr_status sv = validate_create(desc, phys); sv != FR_OK) return sv;
  fr_mesh *m = new (std::nothrow) fr_mesh();
  if (!m) return fail(nullptr, FR_ENOMEM, "host allocation failed");
  if (fr_status st = build_part(desc, part, rank, m->host, m->halo); st != FR_OK) {
    delete m;
    return st;
  }
  m->is_part = true;
  fr_mesh *made = nullptr;
  if (fr_status st = finish_create(m, phys, stream, &made); st != FR_OK) return st;   // m freed on failure
  const HaloLists &halo = made->halo;
  const int64_t n_halo = (int64_t)halo.iface.size();
  if (n_halo > 0) {
    std::vector<int64_t> code((size_t)n_halo);
    for (int64_t k = 0; k < n_halo; ++k) code[k] = 2 * halo.iface[k] + halo.side[k];
    fr_status st = dalloc(made, &made->d_halo, (size_t)n_halo);
    cudaError_t ce = cudaSuccess;
    if (st == FR_OK) {
      ce = cudaMemcpy(made->d_halo, code.data(), code.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
      if (ce != cudaSuccess) st = FR_ECUDA;
    }
    if (st != FR_OK) {
      std::string msg = ce != cudaSuccess ? std::string("halo upload: ") + cudaGetErrorString(ce) : made->err;
      fr_free(made);
      return fail(nullptr, st, msg);
    }
  }
  *out = made;
  return FR_OK;
}

extern "C" fr_status fr_halo_query(const fr_mesh *m, fr_part_info *info, int32_t *peers, int64_t *peer_begin,
                                   int64_t *gid, int64_t *elem_global) {
  if (!m || !info) return FR_EINVAL;
  if (!m->is_part) {
    info->n_elem = m->host.E + m->host.Ep;
    info->n_iface = m->host.n_interior;
    info->n_bface = m->host.n_if - m->host.n_interior;
    info->n_peers = 0;
    info->n_halo = 0;
    if (peer_begin) peer_begin[0] = 0;
    if (elem_global)
      for (int64_t e = 0; e < m->host.E + m->host.Ep; ++e) elem_global[e] = e;
    return FR_OK;
  }
  fill_part_info(m->host, m->halo, info);
  copy_halo(m->halo, peers, peer_begin, gid, elem_global);
  return FR_OK;
}

extern "C" fr_status fr_part_phase(fr_mesh *m, int32_t phase, int32_t scheme, int32_t stage, double t, double dt,
                                   const double *recv_device, double *send_device, double *R_device) {
  (void)t;
  fr_status st = check_mesh(m);
  if (st) return st;
  if (phase < 0 || phase > 2) return fail(m, FR_EINVAL, "phase must be 0, 1 or 2");
  const int64_t n_halo = (int64_t)m->halo.iface.size();
  if (n_halo > 0 && ((phase < 2 && !send_device) || (phase > 0 && !recv_device)))
    return fail(m, FR_EINVAL, "NULL halo buffer");
  DevMesh &d = m->dev;
  const int Nf = d.Nf;
  double *recv = const_cast<double *>(recv_device);
  if (phase == 0) {
    FR_CUDA(m, launch_residual(d, m->dphys, MODE_RESIDUAL, 0, 0.0, nullptr, m->stream, nullptr, 1));
    FR_CUDA(m, launch_halo_copy(d.Qtr, send_device, m->d_halo, n_halo, 5, Nf, 0, m->stream));
    return FR_OK;
  }
  if (phase == 1) {
    FR_CUDA(m, launch_halo_copy(d.Qtr, recv, m->d_halo, n_halo, 5, Nf, 1, m->stream));
    FR_CUDA(m, launch_residual(d, m->dphys, MODE_RESIDUAL, 0, 0.0, nullptr, m->stream, nullptr, 2));
    FR_CUDA(m, launch_halo_copy(d.Gtr, send_device, m->d_halo, n_halo, 15, Nf, 0, m->stream));
    return FR_OK;
  }
  int mode, last;
  switch (scheme) {
    case FR_RESIDUAL_ONLY: mode = MODE_RESIDUAL; last = -1; break;
    case FR_RK44: mode = MODE_RK; last = 3; break;
    case FR_SSPRK33: mode = MODE_SSP33; last = 2; break;
    case FR_SSPRK104: mode = MODE_SSP104; last = 9; break;
    default: return fail(m, FR_EINVAL, "unknown Runge-Kutta scheme");
  }
  if (mode == MODE_RESIDUAL && !R_device) return fail(m, FR_EINVAL, "NULL residual pointer");
  if (mode != MODE_RESIDUAL && (stage < 0 || stage > last || !std::isfinite(dt)))
    return fail(m, FR_EINVAL, "bad stage or dt");
  FR_CUDA(m, launch_halo_copy(d.Gtr, recv, m->d_halo, n_halo, 15, Nf, 1, m->stream));
  FR_CUDA(m, launch_residual(d, m->dphys, mode, mode == MODE_RESIDUAL ? 0 : stage, dt, R_device, m->stream, nullptr,
                             4 | 8));
  if (mode != MODE_RESIDUAL && stage == last) {
    int *hflag = reinterpret_cast<int *>(m->h_scalar);
    FR_CUDA(m, cudaMemcpyAsync(hflag, d.flag, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    FR_CUDA(m, cudaStreamSynchronize(m->stream));
    if (*hflag) {
      const int f = *hflag;
      FR_CUDA(m, cudaMemsetAsync(d.flag, 0, sizeof(int), m->stream));
      if (f & 2) return fail(m, FR_ETIMEOUT, "a tensor-core kernel gave up waiting for its copies or MMAs");
      return fail(m, FR_ENONFINITE, "non-finite value in the updated state");
    }
  }
  return FR_OK;
}

extern "C" const char *fr_last_error(const fr_mesh *m) {
  if (m) return m->err.c_str();
  return g_create_error.c_str();
}

namespace frx {

fr_status frx_mesh_view(fr_mesh *m, DevMesh *dev, DevPhys *phys, cudaStream_t *stream, int *device) {
  fr_status st = check_mesh(m);
  if (st) return st;
  *dev = m->dev;
  *phys = m->dphys;
  *stream = m->stream;
  *device = m->device;
  return FR_OK;
}

fr_status frx_mesh_fail(fr_mesh *m, fr_status st, const std::string &msg) { return fail(m, st, msg); }

bool frx_mesh_has_halo(const fr_mesh *m) { return m && m->is_part && !m->halo.iface.empty(); }

}  // namespace frx
