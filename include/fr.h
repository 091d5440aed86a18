/*
 * fr.h — C ABI of the GB300 flux-reconstruction (FR) library.
 *
 * The library evaluates the semi-discrete FR residual of the compressible Navier–Stokes
 * equations on unstructured hexahedral and mixed hexahedral/prismatic meshes at orders p = 1..7
 * and advances it with explicit
 * Runge–Kutta stages, all on one CUDA device (arXiv 2308.06605, section "FR Algorithm",
 * Eq. 1–3).  Plain C types only; device pointers are raw CUDA pointers, host pointers are plain
 * host memory.  Every call returns an fr_status; nothing aborts.
 *
 * Conventions (all calls):
 *  - Canonical state layout is [element][point][variable], elements in input order, points
 *    m = i + N j + N^2 k (N = p + 1) on ascending Gauss–Legendre nodes along the element's
 *    reference axes xi, eta, zeta, variables (rho, rho u, rho v, rho w, E).  Reference vertex
 *    order of a hexahedron follows VTK/CGNS (bottom face counter-clockwise, then top face).
 *    On meshes with prisms the prism points follow all hexahedral points: prism by prism in
 *    input order, points m = q + Nt k (Nt = N(N+1)/2) with q the triangle node (warp-and-blend
 *    nodes of Warburton 2006 on the reference triangle (-1,-1), (1,-1), (-1,1), enumerated by
 *    barycentric lattice index n = 0..p outer, m = 0..p-n inner) and k the Gauss–Legendre node
 *    along the prism's axis.
 *  - The library copies every host array it is given at create time; pointers passed to other
 *    calls are borrowed for the duration of the call only.
 *  - All device work is enqueued on the stream given to fr_mesh_create (0 = legacy default
 *    stream).  Calls with FR_DEVICE pointers return without synchronising; calls with FR_HOST
 *    pointers synchronise that stream before returning.
 *  - After FR_ECUDA or FR_ETIMEOUT a mesh is poisoned: every later call except fr_free and
 *    fr_last_error returns the same status.
 */
#ifndef FR_H
#define FR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FR_OK = 0,
  FR_EINVAL = 1,        /* bad argument (NULL pointer, out-of-range value) */
  FR_ENOMEM = 2,        /* host or device allocation failed */
  FR_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed (mesh poisoned) */
  FR_EMESH = 4,         /* invalid mesh: unmatched face, unknown tag, non-positive Jacobian */
  FR_EUNSUPPORTED = 5,  /* valid request that this build does not implement */
  FR_ENONFINITE = 6,    /* a non-finite value appeared in the updated state */
  FR_ETIMEOUT = 7       /* a bounded device-side wait expired (mesh poisoned) */
} fr_status;

enum { FR_HOST = 0, FR_DEVICE = 1 };                       /* where a state pointer lives */
enum { FR_RUSANOV = 0, FR_ROE = 1 };                       /* inviscid common flux */
enum { FR_VISC_NONE = 0, FR_VISC_BR2 = 1, FR_VISC_LDG = 2 }; /* viscous treatment */
enum { FR_PREC_FP64 = 0, FR_PREC_MIXED = 1, FR_PREC_MIXED_TC = 2, FR_PREC_MIXED_VF32 = 3 };  /* fr_physics */
enum {                                                     /* explicit Runge–Kutta schemes */
  FR_RK44 = 0,      /* classical four-stage, fourth order */
  FR_SSPRK33 = 1,   /* three-stage third-order SSP (Shu–Osher form), SSP coefficient 1 */
  FR_SSPRK104 = 2   /* Ketcheson's ten-stage fourth-order SSP scheme (two registers), coefficient 6 */
};
enum { FR_RESIDUAL_ONLY = -1 };                            /* fr_part_phase: write R, no stage update */
enum {                                                     /* boundary-condition kinds */
  FR_BC_WALL_ISOTHERMAL = 1,  /* params[0] = wall temperature */
  FR_BC_CHAR_INFLOW = 2,      /* params = total pressure, total temperature, flow direction (3) */
  FR_BC_CHAR_OUTFLOW = 3,     /* params[0] = static pressure */
  FR_BC_DIRICHLET = 4         /* params[0..4] = exterior conserved state */
};

typedef struct fr_mesh fr_mesh;                            /* opaque, owned by the library */

typedef struct {
  int32_t tag;          /* boundary tag as used in fr_mesh_desc.bface_tag */
  int32_t kind;         /* FR_BC_* */
  double params[8];
} fr_bc;

typedef struct {
  int32_t tag_a, tag_b; /* faces tagged tag_b are the faces tagged tag_a translated by t */
  double t[3];
} fr_periodic;

typedef struct {
  int64_t n_nodes;
  const double *xyz;            /* [n_nodes][3] vertex coordinates (host) */
  int64_t n_hex;
  const int64_t *hex;           /* [n_hex][8] vertex ids, VTK order (host) */
  int32_t p;                    /* polynomial order, 1..7, uniform over the mesh */
  int64_t n_bface;
  const int64_t *bface_nodes;   /* [n_bface][4] vertex ids of each boundary face (a triangle
                                   lists three ids and -1) */
  const int32_t *bface_tag;     /* [n_bface] */
  int32_t n_bc;
  const fr_bc *bc;              /* [n_bc] tag -> condition */
  int32_t n_periodic;
  const fr_periodic *periodic;  /* [n_periodic] */
  int64_t n_prism;              /* 0 for a hexahedral mesh */
  const int64_t *prism;         /* [n_prism][prism_nodes] vertex ids, VTK wedge order: (v0, v1, v2)
                                   one triangle, (v3, v4, v5) the opposite one, v_k+3 above v_k (host) */
  int32_t hex_nodes;            /* nodes per hexahedron: 8 (trilinear; 0 means 8) or 27 (triquadratic:
                                   the 8 corners, edge midpoints 01 12 23 30 45 56 67 74 04 15 26 37,
                                   face centres x- x+ y- y+ z- z+, centre) */
  int32_t prism_nodes;          /* nodes per prism: 6 (0 means 6) or 18 (quadratic: the 6 corners,
                                   edge midpoints 01 12 20 34 45 53 03 14 25, centres of the
                                   quadrilateral faces 0143 1254 2035) */
  const int8_t *elem_p;         /* NULL (every element at order p) or [n_hex + n_prism] per-element
                                   orders, hexahedra first (host).  Only uniform orders are built:
                                   an entry outside 1..7 gives FR_EINVAL, an entry that differs from p
                                   FR_EUNSUPPORTED (interfaces between elements of different orders
                                   are not built; ensembles of different orders run as batches) */
} fr_mesh_desc;

typedef struct {
  double gamma;         /* ratio of specific heats */
  double R;             /* gas constant (p = rho R T) */
  double mu;            /* dynamic viscosity (constant) */
  double Pr;            /* Prandtl number */
  int32_t inviscid;     /* FR_RUSANOV (local Lax-Friedrichs) | FR_ROE (Roe average, Harten's entropy
                           fix on the acoustic waves with delta = 0.1 c); FP64 on both precisions */
  int32_t viscous;      /* FR_VISC_NONE | FR_VISC_BR2 */
  double br2_eta;       /* BR2 penalty factor (number of faces, 6, by default) */
  int32_t precision;    /* FR_PREC_FP64 | FR_PREC_MIXED: element operators (traces, gradients,
                           fluxes at solution points, divergence, correction) in double-float
                           (FP32 hi + lo pairs); Riemann flux, boundary states and RK in FP64 |
                           FR_PREC_MIXED_TC: as FR_PREC_MIXED, with the face interpolation (Eq. 2,
                           the solution at the flux points) on the tensor cores: tcgen05.mma in
                           TF32 with FP32 accumulation on exponent-aligned 10-bit slices of the
                           data and of l(+-1) (error-free splitting, Ozaki et al. 2012), 5 slices
                           each, combined into double-float; error at most 2^-44 of the line's
                           largest value times max |l| (hexahedra; not in fr_batch_create:
                           FR_EUNSUPPORTED) |
                           FR_PREC_MIXED_VF32: as FR_PREC_MIXED, with the viscous branch of the
                           hexahedral volume kernel (corrected gradients of the perturbation from
                           the element's first point, gradient traces, stress and heat flux) and
                           the interface viscous flux in plain FP32.  Its error is FP32 rounding of
                           the viscous terms amplified by the second derivative: about 1e-6 of the
                           viscous part of the residual, so relative to the residual it grows
                           like 1/Re and with the viscous share (measured normwise <= 7.7e-7 per
                           variable on perturbed TGV states at Re >= 400, p <= 7; 2.1e-6 at the
                           initial TGV state at Re 1600, whose residual is almost purely viscous;
                           1e-5 at Re = 20).  c = 0 only (FR_EUNSUPPORTED otherwise); prisms keep
                           double-float; not in fr_batch_create */
  double ldg_tau;       /* LDG penalty tau (FR_VISC_LDG): at each interface the side whose face
                           normal (summed over the face) points along (1, sqrt2/2, sqrt3/4)
                           supplies the common solution, the other side the common gradient
                           (corrected gradients interpolated to the face), and the common
                           normal flux gains tau |n| (Q_0 - Q_1) (boundaries: tau |n| (Q- - Q_b)) */
  double vcjh_c;        /* correction function (section "FR Algorithm"): 0 is the paper's
                           DG-equivalent choice (right/left Radau polynomials); c != 0 selects the
                           member c of the energy-stable family of Vincent, Castonguay & Jameson
                           (2011), g_L = (-1)^p/2 [P_p - (eta P_{p-1} + P_{p+1}) / (1 + eta)],
                           eta = c (2p+1) (a_p p!)^2 / 2, a_p = (2p)! / (2^p (p!)^2); the same
                           correction fields correct the gradient of the viscous terms.  Needs
                           1 + eta > 0 (FR_EINVAL otherwise); c != 0 is built for hexahedral meshes
                           on the per-mesh path (fr_mesh_create with prisms, fr_batch_create and
                           fr_residual_static return FR_EUNSUPPORTED) */
} fr_physics;

typedef struct {
  int64_t n_elem;       /* elements */
  int32_t p, n_pts;     /* order and solution points per element ((p+1)^3) */
  int64_t n_iface;      /* interior + periodic interfaces */
  int64_t n_bface;      /* boundary-condition faces */
  int64_t device_bytes; /* device memory held by the mesh */
  int64_t n_prism;      /* prisms (after the n_elem hexahedra in every per-point array) */
  int32_t n_pts_prism;  /* solution points per prism: (p+1)(p+2)/2 triangle nodes x (p+1) */
  int64_t n_points;     /* all solution points: n_elem n_pts + n_prism n_pts_prism */
  int32_t device;       /* CUDA device the mesh lives on (fr_mesh_query; -1 from fr_mesh_inspect) */
} fr_mesh_info;

/*
 * fr_mesh_create — build connectivity, geometry and device buffers (section "FR Algorithm",
 * Eq. 1: |J| and S = |J| J^-1 at the solution points; the paper's face construction: faces are
 * keyed by their sorted vertex ids (corners), sorted so coupled faces are adjacent, then paired).
 * Quadratic (curved) elements take their metric terms from the conservative curl form (Kopriva
 * 2006): S[i][n] = -(curl I(X_l grad X_m))_i, (n, m, l) cyclic, I the degree-p interpolant on
 * Gauss-Lobatto points (on the prism: triangle nodes x Gauss-Lobatto in zeta), evaluated exactly
 * at the solution and flux points, so free stream is preserved to rounding; linear elements use
 * the analytic S.
 * Periodic faces are paired by translated centroids.  Validates everything before allocating
 * device memory: unmatched interior faces, boundary faces without a condition, non-positive
 * Jacobians -> FR_EMESH; p outside 1..7, NULL arrays, bad physics -> FR_EINVAL.  `stream` is a
 * cudaStream_t cast to uintptr_t.  On success *out owns all device memory until fr_free.
 */
fr_status fr_mesh_create(const fr_mesh_desc *desc, const fr_physics *phys, uintptr_t stream,
                         fr_mesh **out);

/*
 * fr_mesh_inspect — the host half of fr_mesh_create without any device work: validates the
 * description and builds connectivity and geometry (same checks and statuses as fr_mesh_create
 * for the mesh itself), then fills *info (device_bytes = 0) and, where the pointers are not NULL,
 * the solution points xyz_host [n_points][3] in the canonical order and the metric terms
 * metrics_host: hexahedra [n_elem][10][n_pts] then prisms [n_prism][10][n_pts_prism], per point
 * S = |J| J^-1 row-major (reference direction, physical component) and then 1/|J| (Eq. 1);
 * the hexahedra's face table ef_host [n_elem][6] (interface << 4 | side << 3 | orientation
 * code; faces ordered xi-, xi+, eta-, eta+, zeta-, zeta+; interfaces: the n_iface two-sided ones,
 * then the boundary faces) and normals_host [n_iface + n_bface][4][(p+1)^2]: side 0's outward
 * area-scaled normal at each flux point in side 0's point order, then its length.  A face point
 * (a, b) of either side sits in slot a' + (p+1) b' with (a', b') = (b, a) if code & 4, then a'
 * reversed if code & 1 and b' reversed if code & 2 (side 0 carries code 0).  Prisms: ef_prism_host [n_prism][5] packed the same way
 * (faces zeta-, zeta+ (triangles), then s = -1, r + s = 0, r = -1 (quadrilaterals, points
 * a + (p+1) b with a along the edge and b along zeta)); a triangular face's node q sits in slot
 * tri_slot_host[code][q] ([6][(p+1)(p+2)/2], code 0 the identity).  Call once with NULL arrays for
 * the sizes.  Caller-owned host buffers.
 */
fr_status fr_mesh_inspect(const fr_mesh_desc *desc, fr_mesh_info *info, double *xyz_host, double *metrics_host,
                          int32_t *ef_host, double *normals_host, int32_t *ef_prism_host, int32_t *tri_slot_host);

/* fr_mesh_query — sizes of a created mesh (host struct filled). */
fr_status fr_mesh_query(const fr_mesh *mesh, fr_mesh_info *info);

/*
 * fr_solution_points — physical coordinates of the solution points, [n_points][3] in the
 * canonical order, written to host memory (Eq. 2: the nodal points of the element map).
 */
fr_status fr_solution_points(fr_mesh *mesh, double *xyz_host);

/*
 * fr_basis_1d — the 1D tables of order p that the element kernels apply along each reference
 * line (Eq. 2 and the correction term of Eq. 3), computed on the host, no device work: the
 * N = p + 1 Gauss-Legendre nodes x and weights w, the nodal derivative matrix D[i*N + a] =
 * l_a'(x_i), the boundary values lm[a] = l_a(-1), lp[a] = l_a(+1), and the correction
 * divergences hm[i] = g_R'(-x_i), hp[i] = g_R'(x_i) of the correction function with parameter c
 * (vcjh_c of fr_physics; 0 = DG-equivalent).  Arrays are caller-owned host buffers of N (D:
 * N*N) doubles; any of them may be NULL.  p outside 1..7 or c outside the family -> FR_EINVAL.
 */
fr_status fr_basis_1d(int32_t p, double c, double *x, double *w, double *D, double *lm, double *lp,
                      double *hm, double *hp);

/*
 * fr_tri_basis — the nodal triangle tables of order p that the prism kernels apply (host
 * computation, no device work): the Nt = (p+1)(p+2)/2 warp-and-blend nodes rs[Nt][2] in the
 * canonical prism order, the derivative matrices Dr, Ds [Nt][Nt] and the inverse mass matrix
 * Minv [Nt][Nt] of the nodal basis.  Caller-owned host buffers, any may be NULL; p outside 1..7
 * -> FR_EINVAL.
 *
 * fr_transfer_matrix — the L2-projection operator of fr_project_state from order p to order q
 * (host computation): kind 0 the line [q+1][p+1] (Legendre coefficients through the Gauss
 * points, truncated or zero-padded), kind 1 the triangle [Nt_q][Nt_p] (orthonormal modes of
 * total degree <= min(p, q)).  p, q in 1..7, else FR_EINVAL.
 */
fr_status fr_tri_basis(int32_t p, double *rs, double *Dr, double *Ds, double *Minv);
fr_status fr_transfer_matrix(int32_t kind, int32_t p, int32_t q, double *T);

/*
 * fr_set_state / fr_get_state — copy the solution Q (canonical layout, n_points*5 doubles)
 * into / out of the mesh.  `where` = FR_HOST or FR_DEVICE.  fr_set_state also resets the
 * Runge–Kutta registers (the solution becomes the start of a new step).
 */
fr_status fr_set_state(fr_mesh *mesh, const double *Q, int32_t where);

/*
 * fr_project_state — set dst's state to the L2 projection of src's current state onto dst's order
 * (the paper starts at low order and switches to a higher one).  src and dst describe the same
 * elements (same mesh description, any two orders); in reference coordinates the projection keeps
 * the Legendre modal coefficients on each hexahedron axis, and the orthonormal triangle modes times
 * Legendre on prisms, up to the lower of the two degrees.  Waits for src's stream, works on dst's
 * and returns when done; dst's Runge-Kutta registers restart from the projected state.  Different
 * element counts or devices -> FR_EINVAL.
 */
fr_status fr_project_state(fr_mesh *src, fr_mesh *dst);
fr_status fr_get_state(fr_mesh *mesh, double *Q, int32_t where);

/*
 * fr_residual — R = dQ/dt of the current state (Eq. 3: -|J|^-1 [div_xi F^ + sum over faces and
 * flux points of div(g) (F^I_perp - F_perp)] with the DG-equivalent correction, the Rusanov or
 * Roe common flux and the BR2 viscous flux), written in the canonical layout to R (FR_HOST or
 * FR_DEVICE).  `t` is the physical time (used by time-dependent boundary data).
 */
fr_status fr_residual(fr_mesh *mesh, double t, double *R, int32_t where);

/*
 * fr_rk_stage — one stage of the explicit Runge–Kutta scheme (the paper advances Eq. 3 with an
 * explicit RK method; this library provides classical RK44).  Stage k in 0..3 evaluates the
 * residual of the current stage state at time t + c_k dt and updates, in FP64,
 *   acc += b_k dt R,  U = U_n + a_{k+1} dt R       (k < 3)
 *   U_n = U_n + acc + b_3 dt R,  U = U_n           (k = 3)
 * with a = (1/2, 1/2, 1), b = (1/6, 1/3, 1/3, 1/6).  acc and U_n are FP64 in both precisions;
 * with FR_PREC_MIXED the intermediate stage state U is held only as double-float for the element
 * kernels, so fr_get_state between stages returns U_n (the state of the last completed step).
 * Stages must be called in order 0,1,2,3;
 * `t` is the time at the start of the step.  Returns FR_ENONFINITE (checked at stage 3 only) if
 * a non-finite value was written.
 * The paper names strong-stability-preserving RK (Ketcheson 2008) as its integrator; two are
 * built, with FP64 registers on both precisions (U_n, the stage state U, and acc):
 *   FR_SSPRK33  stages 0..2:  U = a_k U_n + b_k (U + dt R), (a, b) = (0, 1), (3/4, 1/4), (1/3, 2/3)
 *   FR_SSPRK104 stages 0..9:  U = U + dt/6 R (stages 0..8); after stage 4, q2 = U_n/25 + 9/25 U is
 *               kept in acc and U = 15 q2 - 5 U; stage 9: U = q2 + 3/5 U + dt/10 R.
 * At the last stage U_n = U and non-finite values are reported.  Between stages fr_get_state
 * returns the stage state U for these schemes (on both precisions).
 */
fr_status fr_rk_stage(fr_mesh *mesh, int32_t scheme, int32_t stage, double t, double dt);

/*
 * fr_max_dt — dt = cfl * min_e h_e / ((2p + 1) max over the element's points of (|u| + c)),
 * h_e = volume^(1/3): an explicit-stability estimate (not specified by the paper).
 */
fr_status fr_max_dt(fr_mesh *mesh, double cfl, double *dt);

/*
 * Domain decomposition (paper, section "Pre-processing": the mesh is distributed over processes,
 * the faces on partition boundaries are paired (Algorithm 2, "MatchMPIFaces"), and every step
 * exchanges the data of those faces).  Hexahedral and mixed hexahedral/prismatic meshes.  A part
 * holds its own elements and every interface touching them; an interface shared with another
 * part (a halo interface) keeps the global mesh's record, so each part writes its own side's
 * traces and receives the other side's from the peer.  BR2 and LDG are compact, so one exchange of solution traces (before the
 * volume kernel needs the jumps) and one of gradient traces (before the interface fluxes) per
 * stage make each part's residual equal to the residual of the whole mesh restricted to the part.
 */
typedef struct {
  int64_t n_elem;       /* elements of the part */
  int64_t n_iface;      /* two-sided interfaces touching them (including halo interfaces) */
  int64_t n_bface;      /* boundary-condition faces of the part */
  int32_t n_peers;      /* parts sharing interfaces with this one */
  int64_t n_halo;       /* halo interfaces */
} fr_part_info;

/*
 * fr_partition — host only: recursive coordinate bisection of the element centroids (mean of the
 * corner vertices) into n_parts parts of near-equal solution-point count; each cut is across the
 * longest extent, ties ordered by element index, so the result is deterministic.  part: [n_hex +
 * n_prism] caller-owned host array, written with ids 0..n_parts-1 (elements in input order).
 * FR_EINVAL for n_parts < 1 or > the element count, FR_EMESH for a vertex id out of range.
 */
fr_status fr_partition(const fr_mesh_desc *desc, int32_t n_parts, int32_t *part);

/*
 * fr_partition_cost — fr_partition with each element weighted by its solution points times the
 * cost of one point of its type: cost_hex for hexahedra, cost_prism for prisms (any positive unit,
 * e.g. the measured time per point of each type at this order and arithmetic, or the algorithmic
 * flops per point), so parts of mixed meshes balance work rather than points.  FR_EINVAL for a
 * cost that is not finite and positive; otherwise as fr_partition.
 */
fr_status fr_partition_cost(const fr_mesh_desc *desc, int32_t n_parts, double cost_hex, double cost_prism,
                            int32_t *part);

/*
 * fr_part_inspect — host only: what fr_mesh_create_part would build for part `rank` (no device
 * work).  info is filled; each array may be NULL: peers [n_peers] (ascending), peer_begin
 * [n_peers + 1] (halo entries of peer k are [peer_begin[k], peer_begin[k+1])), gid [n_halo] (the
 * global interface number of each halo entry; ascending within a peer), elem_global [n_elem] (the
 * input index of each local element; local elements are in input order: the part's hexahedra,
 * then its prisms).  The halo entries a part sends to a peer and those the peer receives from it
 * are the same interfaces in the same order.  FR_EINVAL for a negative part id or an empty part.
 */
fr_status fr_part_inspect(const fr_mesh_desc *desc, const int32_t *part, int32_t rank, fr_part_info *info,
                          int32_t *peers, int64_t *peer_begin, int64_t *gid, int64_t *elem_global);

/*
 * fr_mesh_create_part — the mesh of part `rank` of the partition `part` ([n_hex + n_prism] host
 * array, ids >= 0), on the current device.  States, residuals and fr_solution_points are in the part's local
 * element order (elem_global of fr_halo_query maps them to input indices).  A part without halo
 * interfaces behaves like fr_mesh_create; a part with them runs its stages through fr_part_phase
 * (fr_residual, fr_rk_stage, fr_residual_static and fr_batch_create return FR_EUNSUPPORTED for it)
 * and refuses the eddy-viscosity closure (the remote elements' eddy viscosity is not exchanged).
 * fr_max_dt is the part's own minimum (reduce it over the parts).
 */
fr_status fr_mesh_create_part(const fr_mesh_desc *desc, const fr_physics *phys, const int32_t *part, int32_t rank,
                              uintptr_t stream, fr_mesh **out);

/* fr_halo_query — the part's sizes and halo lists, as fr_part_inspect (any array may be NULL). */
fr_status fr_halo_query(const fr_mesh *mesh, fr_part_info *info, int32_t *peers, int64_t *peer_begin, int64_t *gid,
                        int64_t *elem_global);

/*
 * fr_part_phase — one third of a residual evaluation or RK stage of a part, enqueued on the mesh's
 * stream.  Halo buffers are caller-owned device arrays of n_halo entries, entry k holding
 * nv x (p+1)^2 8-byte values (nv = 5 solution, 15 gradient; FP64 or, on FR_PREC_MIXED meshes,
 * double-float pairs: the caller only moves them).  Between phases the caller moves the entries of
 * peer k ([peer_begin[k], peer_begin[k+1]) of its send buffer) into that peer's receive buffer at
 * the peer's entries for this part (same count, same order), after the phase's work is complete
 * on the stream.
 *   phase 0: face traces and boundary states; writes the solution halo to send_device (nv = 5).
 *   phase 1: reads the received solution halo from recv_device, runs the volume kernel, writes the
 *            gradient halo to send_device (nv = 15).
 *   phase 2: reads the received gradient halo from recv_device, interface and boundary fluxes,
 *            correction; scheme = FR_RESIDUAL_ONLY writes R to R_device ([n_elem][n_pts][5] device)
 *            at the current state, otherwise applies stage `stage` of the scheme with step dt as
 *            fr_rk_stage does (FR_ENONFINITE at the last stage).
 * A part without halo interfaces may pass NULL buffers.  FR_EINVAL for a bad phase, stage, scheme
 * or NULL pointer.
 */
fr_status fr_part_phase(fr_mesh *mesh, int32_t phase, int32_t scheme, int32_t stage, double t, double dt,
                        const double *recv_device, double *send_device, double *R_device);

/*
 * fr_residual_static — the residual of a caller-supplied state, computed without allocating
 * anything.  (The paper has no counterpart: this is a deployment variant of fr_residual.)
 *
 * For callers that cannot allocate device memory when they need a residual: code embedded in
 * another framework that owns the device's memory pool, loops that must not hit cudaMalloc's
 * implicit device synchronisation, or plug-ins that are only handed existing buffers.  The
 * intermediate arrays of the residual (face traces, gradient traces, common fluxes, partial
 * residual) live in one static device array of 32 MiB that every device loading this library
 * holds until the process exits; no cudaMalloc, cudaFree or allocating library routine is
 * called.  Q_device (input, [n_elem][n_pts][5] canonical layout) and R_device (output, same
 * layout) are caller-owned device pointers on the mesh's device, which must be the current
 * device (otherwise FR_EINVAL, and the mesh stays usable); the mesh's state arrays are not read
 * or changed (its geometry and connectivity are read).
 * Meshes whose intermediates exceed 32 MiB (8 bytes x (45 n_iface_total N^2 + 5 n_elem N^3),
 * N = p + 1) are rejected with FR_EINVAL and a message giving both sizes.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) — make that first call
 * before any stream capture.  All calls share the one array and it keeps the last call's
 * contents; nothing in it needs to start at zero, but calls whose work overlaps on the GPU
 * (other streams, other meshes, other threads) race on it: serialise them.  Work is enqueued
 * on the mesh's stream and the call returns without synchronising.  FP64 hexahedral meshes with
 * the DG-equivalent correction (c = 0) and without the eddy-viscosity closure only
 * (FR_EUNSUPPORTED for FR_PREC_MIXED, a mesh with prisms, c != 0 or the closure switched on).
 */
fr_status fr_residual_static(fr_mesh *mesh, const double *Q_device, double *R_device);

/*
 * Eddy-viscosity closure (the paper lists LES sub-grid-scale models among its physical models;
 * this is a learned one).  Per element, a network of 11 -> 64 -> 64 -> 64 -> 1 (GELU, softplus
 * output) maps the features x = (element-mean corrected velocity gradient du_i/dx_j, 9 values
 * row-major; |S| = sqrt(2 S_ij S_ij); Delta = h/(p+1)) to nu_t = s_out Delta^2 softplus(z); the
 * viscous fluxes use mu + rho nu_t and kappa + rho nu_t cp / Pr_t (Pr_t = 0.9), with the mean of the
 * two elements' nu_t at interfaces.  params: FR_CLOSURE_NPARAMS floats, layout W1[64][11], b1[64],
 * W2[64][64], b2[64], W3[64][64], b3[64], w4[64], b4[1]; stored on the device as bfloat16 (round to
 * nearest even) and evaluated with FP32 accumulation inside the volume kernel.  scales: 23 floats
 * (input mean[11], input std[11], s_out).  enable = 0 switches it off.  Needs the viscous path;
 * hexahedral meshes only (FR_EUNSUPPORTED on a mesh with prisms); not available in batches.  fr_closure_nu copies the last evaluated nu_t per element to the host.
 */
#define FR_CLOSURE_NPARAMS 9153
#define FR_CLOSURE_PRT 0.9
fr_status fr_set_closure(fr_mesh *mesh, const float *params, const float *scales, int32_t enable);

/*
 * fr_set_source — the source term S of Eq. 3 (the paper's body forcing and sponge zones near
 * inflow and outflow), added to the residual at every solution point in FP64:
 *   body acceleration g (accel[3], NULL = off):  S = (0, rho g, rho u . g)
 *   sponge (sigma [n_points] >= 0 and Q_ref [n_points][5], canonical order, both NULL = off):
 *                                                S = -sigma (Q - Q_ref)
 * evaluated on the state the residual is computed from (the stage state in RK stages).  Host
 * arrays are copied; a later call replaces the previous settings.  sigma without Q_ref (or the
 * reverse), negative or non-finite values -> FR_EINVAL.  A batch uses the settings its meshes had
 * when fr_batch_create was called.
 */
fr_status fr_set_source(fr_mesh *mesh, const double *accel, const double *sigma, const double *Q_ref);
fr_status fr_closure_nu(fr_mesh *mesh, float *nu_host);

/*
 * Training kernels of the closure network (FP32; all pointers are device pointers, work is
 * enqueued on `stream` and the calls return without synchronising).  X: [n][11] raw features,
 * scales as in fr_set_closure (only mean/std are used), y: [n] targets of softplus(z) (that is
 * nu_t / (s_out Delta^2)).  work: fr_mlp_workspace_floats(n) floats owned by the caller.
 * fr_mlp_forward writes softplus(z) to out[n].  fr_mlp_loss_grad writes the mean squared error to
 * *loss and its gradient with respect to every parameter to grad[FR_CLOSURE_NPARAMS].
 * fr_mlp_adam applies one Adam update (Kingma & Ba 2015) with bias correction for step >= 1.
 */
int64_t fr_mlp_workspace_floats(int64_t n);
fr_status fr_mlp_forward(const float *params, const float *scales, const float *X, int64_t n, float *out, float *work,
                         uintptr_t stream);
fr_status fr_mlp_loss_grad(const float *params, const float *scales, const float *X, const float *y, int64_t n,
                           float *grad, float *loss, float *work, uintptr_t stream);
fr_status fr_mlp_adam(float *params, const float *grad, float *m, float *v, int32_t n_params, float lr, float beta1,
                      float beta2, float eps, int32_t step, uintptr_t stream);

/*
 * Batched stages for ensembles of independent cases (the paper runs one mesh per MPI
 * decomposition; on one GPU an ensemble of unevenly sized cases, with different orders, is
 * advanced together).  fr_batch_create borrows the meshes (they must outlive the batch, share
 * precision, device and stream; meshes may mix hexahedra and prisms, of any geometry order; meshes
 * with the closure are rejected with FR_EUNSUPPORTED).  fr_batch_rk_stage runs stage `stage` (RK44, same update as
 * fr_rk_stage) of every case in ONE cooperative persistent kernel: phases (face interpolation,
 * boundary states, volume, interface fluxes, correction + update) are separated by grid
 * barriers whose waits are bounded; if a wait gives up, the call returns FR_ETIMEOUT and the
 * batch and its meshes are poisoned.  On a non-default stream each stage is captured once into
 * a CUDA graph and replayed.  Errors (timeout, non-finite values) are read back at stage 3.
 * fr_batch_set_dt sets each case's step size (host array, one per case).  fr_batch_tune times
 * the persistent kernel's block size (256/512 threads, which fixes the elements-per-block tile of
 * every order) and resident blocks per SM, and the alternative executor -- every case's own
 * order-specialised kernels captured back to back in one graph per stage -- keeps the fastest
 * (fr_batch_info.mode: 0 persistent, 1 per-case kernels), and restores every case to its U_n.  fr_batch_debug (tests only) makes block `skip_block` leave before its first barrier,
 * with a barrier wait limit of `spin_limit` iterations, to exercise the timeout path.
 */
typedef struct fr_batch fr_batch;
typedef struct {
  int32_t n_cases, block, grid, blocks_per_sm;
  int64_t n_points, smem_bytes;
  int32_t n_tasks;
  int32_t mode;          /* 0: one persistent cooperative kernel per stage; 1: per-case kernels */
} fr_batch_info;
fr_status fr_batch_create(fr_mesh *const *meshes, int32_t n, fr_batch **out);
fr_status fr_batch_set_dt(fr_batch *batch, const double *dt_host);
fr_status fr_batch_rk_stage(fr_batch *batch, int32_t stage, double t);
fr_status fr_batch_tune(fr_batch *batch);
fr_status fr_batch_query(const fr_batch *batch, fr_batch_info *info);
/* fr_batch_select — force the executor: 0 persistent cooperative kernel, 1 per-case kernels. */
fr_status fr_batch_select(fr_batch *batch, int32_t mode);
fr_status fr_batch_debug(fr_batch *batch, int32_t skip_block, int64_t spin_limit);
void fr_batch_free(fr_batch *batch);
const char *fr_batch_last_error(const fr_batch *batch);

/*
 * Instrumentation (not part of the method).  fr_profile(mesh, 1) makes every later residual
 * evaluation record CUDA events around each of its kernels on the mesh's stream;
 * fr_profile_read accumulates, per kernel k < n, the summed device time in milliseconds
 * (ms[k]) and the number of launches (launches[k]) since profiling was enabled, synchronising
 * the stream first.  Kernel order: 0 face interpolation, 1 volume, 2 interface flux,
 * 3 correction + update.  fr_profile(mesh, 0) stops recording and clears the totals.
 */
#define FR_N_KERNELS 4
fr_status fr_profile(fr_mesh *mesh, int32_t enable);
fr_status fr_profile_read(fr_mesh *mesh, double *ms, int64_t *launches, int32_t n);

/* fr_free — release all host and device memory of the mesh (NULL-safe). */
void fr_free(fr_mesh *mesh);

/* fr_last_error — human-readable message of the last failing call on `mesh` (or of the last
 * failing fr_mesh_create when mesh is NULL).  Owned by the library. */
const char *fr_last_error(const fr_mesh *mesh);

#ifdef __cplusplus
}
#endif

#endif /* FR_H */
