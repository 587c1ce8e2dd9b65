/*
 * fr_gb300.h -- C ABI of the GB300 (sm_103a) flux-reconstruction library.
 *
 * The library evaluates the right-hand side (RHS) R(u) of the semi-discrete system du/dt = R(u)
 * obtained by flux reconstruction (FR) of the compressible Navier-Stokes equations with flux
 * anti-aliasing, on hexahedral (affine or trilinear), prismatic, tetrahedral and pyramidal meshes,
 * and advances it with classical RK4.
 * Paper: Akkurt, Witherden, Vincent, "Cache blocking for flux reconstruction: extension to
 * Navier-Stokes equations and anti-aliasing".
 *   - governing equations, fluxes and the perfect-gas closure: Sec. 2.1 (Eqs. gov, fluxe, fluxv);
 *   - the FR steps (disu, con_u, corrected gradient, tdisf, common fluxes, corrected divergence):
 *     Sec. 2.1 Eqs. FR-disu .. FRfinal, and their kernel form in Sec. 2.2;
 *   - flux anti-aliasing (interpolation to quadrature points, L2 projection): Sec. 2.1.1 and
 *     Sec. 2.2.1 (operators M7..M10); sum factorisation of the hex and prism operators: Sec. 4;
 *     tetrahedra and pyramids (listed in Sec. 1 among the supported types) with dense per-element
 *     operators;
 *   - the semi-discrete form du/dt = -J^-1 div~ f~: Eq. govqtrans; RK4: Sec. 3.
 *
 * Conventions shared by every entry point
 *   - Status: every call returns an fr_status; FR_OK is 0. Argument and mesh errors are reported
 *     synchronously and leave the handle unchanged. Device-side conditions (a non-physical state:
 *     rho <= 0, p <= 0 or a non-finite value met while evaluating fluxes) are latched in a device
 *     status word and reported as FR_ENONPHYS by fr_sync_status() or by the next call on the
 *     handle once the earlier work has completed. No call aborts, traps or exits.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     RHS and RK4 calls are asynchronous with respect to the host. A handle may be used by one
 *     stream at a time.
 *   - Ownership: the library copies the host mesh descriptors and owns every device buffer it
 *     allocates (geometry, operators, connectivity, face arrays, RK4 registers). The caller owns
 *     the state U and the result R: device pointers (or host pointers for the *_host variants).
 *   - Layout of U and R (reading R10 of the design notes): element-major [elem][var][pt], with
 *     var in (rho, rho vx, rho vy, rho vz, E). Elements are ordered instance by instance; inside an
 *     instance hexahedra come first, then prisms, then tetrahedra, then pyramids, each in descriptor
 *     order. Hex
 *     point index is i + n j + n^2 k (n = p+1 Gauss-Legendre points per direction, i fastest along
 *     xi); prism point index is t + 10 k (t = triangle point in the paper's printed Williams-Shunn
 *     order, k = Gauss-Legendre level in z); tetrahedron point index runs over the order-3 lattice
 *     points (a, b, c), a + b + c <= 3, a fastest, then b, then c, each at reference coordinates
 *     -1/2 + 4/5 (-1 + 2 (a, b, c)/3 + 1/2) (the lattice shrunk by 4/5 towards the centroid);
 *     pyramid point index runs over the order-3 pyramid lattice, layer k = 0..3 at z = -1 + 2k/3
 *     with (4-k)^2 points x, y = (1 - k/3)(-1 + 2i/(3-k)) (i fastest, then j, then k), shrunk by
 *     4/5 towards (0, 0, -1/2).
 *   - Element type of U/R: double for FR_FP64; float for FR_FP32 and the mixed forms. The RK4
 *     entry points always take an FP64 master state (double), whatever the compute precision.
 *   - Vertex order: hexahedra in tensor order (corner a + 2b + 4c for (a,b,c) in {0,1}^3);
 *     prisms v0,v1,v2 at the lower triangle mapped to the reference (-1,-1),(1,-1),(-1,1) and
 *     v3,v4,v5 above them; tetrahedra v0..v3 mapped to the reference (-1,-1,-1), (1,-1,-1),
 *     (-1,1,-1), (-1,-1,1); pyramids: the base corners in tensor order, reference (-1,-1,-1),
 *     (1,-1,-1), (-1,1,-1), (1,1,-1), then the apex, reference (0,0,1). Prisms, tetrahedra and
 *     pyramids must be affine (other ones give FR_EUNSUPPORTED); a non-affine hexahedron is a
 *     trilinear (curved) element.
 *   - Local face order (used by the L/R rule): hex -xi, +xi, -eta, +eta, -zeta, +zeta; prism
 *     z=-1 triangle, z=+1 triangle, y=-1 quad, x+y=0 quad, x=-1 quad; tetrahedron z=-1, y=-1,
 *     x=-1, x+y+z=-1 (each with the 10 printed triangle points as flux points); pyramid base z=-1
 *     (4 x 4 GL points), then the triangles y=-(1-z)/2, x=(1-z)/2, y=(1-z)/2, x=-(1-z)/2.
 */
#ifndef FR_GB300_H
#define FR_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FR_OK = 0,
    FR_EINVAL = 1,        /* bad argument */
    FR_ENOMEM = 2,        /* device or host allocation failed */
    FR_ECUDA = 3,         /* a CUDA runtime call failed (text in fr_last_error()) */
    FR_EMESH = 4,         /* non-conforming mesh: unmatched face or flux point, inverted element */
    FR_ETIMEOUT = 5,      /* a bounded device wait gave up (the tensor-core completion wait of the
                           * mixed forms; latched on the device like FR_ENONPHYS) */
    FR_ENONPHYS = 6,      /* non-physical state met on the device */
    FR_EUNSUPPORTED = 7,  /* valid request outside what this build implements */
    FR_EBOUNDS = 8        /* the bounds-checking build (compiled with FR_DEBUG_BOUNDS) met an element
                           * offset or partner index outside the handle's arrays; the access was
                           * skipped (latched on the device like FR_ENONPHYS) */
} fr_status;

typedef enum {
    FR_FP64 = 0,          /* all arithmetic in FP64 */
    FR_FP32 = 1,          /* FP32 state, operators and fluxes */
    FR_MIXED_BF16 = 2,    /* FR_FP32, except that the dense prism triangle-plane interpolation and
                           * projection (Sec. 4.1 factorisation; the M7 and M8 triangle blocks) run
                           * on the tensor cores as split products with FP32 accumulation: each
                           * operand in three bf16 terms, x = x1 + x2 + x3, and the six products
                           * x1 y1 + x1 y2 + x2 y1 + x1 y3 + x2 y2 + x3 y1 (about 24 significant
                           * bits; two bf16 terms keep only about 16). Hexahedra run the FR_FP32
                           * kernels (their sum-factorised 1D operators are not dense contractions)
                           * unless fr_set_hex_tensor_cores() is on; tetrahedra and pyramids run
                           * the FR_FP32 kernels unless fr_set_dense_tensor_cores() is on. */
    FR_MIXED_FP16 = 3     /* as FR_MIXED_BF16 with fp16 halves, x = x_hi + x_lo, and the three
                           * products x_hi y_hi + x_lo y_hi + x_hi y_lo; every operand row is
                           * scaled by a power of two first (removed exactly afterwards) so that
                           * fp16 keeps its full precision in the low half */
} fr_precision;

typedef enum {
    FR_FUSED = 0,         /* three launches per RHS: face solution, volume group, interface group */
    FR_UNFUSED = 1        /* one kernel per paper kernel (13 launches per RHS), global intermediates */
} fr_form;

/* Physical and discretisation parameters of one instance. */
typedef struct {
    double gamma;         /* ratio of specific heats */
    double Pr;            /* Prandtl number */
    double mu;            /* dynamic viscosity (constant) */
    double beta;          /* LDG switch (Sec. 2.1 common solution and viscous flux) */
    double tau;           /* LDG penalty */
    int p;                /* solution order; hex p in {3,4}, prism, tetrahedron and pyramid p = 3 */
    int nq1d;             /* Gauss-Legendre quadrature points per line: 0 or p + 2 = flux anti-aliasing
                           * (Sec. 2.2.1; tetrahedra: the collapsed (p+2)^3 Gauss-Jacobi rule, exact
                           * to degree 2p+3); p + 1 = no anti-aliasing, the flux is evaluated at the
                           * solution points (the collocation form; hexahedra, fused form only) */
    int tri_strength;     /* prism triangle quadrature strength (0 = 8); collapsed k x k rule, k = strength/2 + 1 */
    int prec;             /* fr_precision */
    int rusanov_mode;     /* 0: wave speed max(|vL.n|+cL, |vR.n|+cR) (the only mode implemented) */
    double p_ref;         /* constant reference pressure removed from the momentum flux, in the volume
                           * and at interfaces (0 = none). On affine elements this changes the RHS only
                           * by rounding: a constant flux has zero divergence and its common flux
                           * equals its own normal flux. It keeps the O(1/(gamma M^2)) pressure out of
                           * the rounding of the momentum divergence. */
    double rho_ref;       /* reference density. With p_ref > 0 and rho_ref > 0 the FP32 form works on
                           * deviations from the reference state (rho_ref, 0, 0, 0, p_ref/(gamma-1)),
                           * evolves the reduced energy E - H0 rho (H0 = gamma p_ref/((gamma-1) rho_ref))
                           * in FP32 and the mass equation in float-float (about 48 bits), then
                           * returns R_E = R_(E-H0 rho) + H0 R_rho. All of it is exact in exact
                           * arithmetic; it removes the O(1/M^2) cancellations of low-Mach flows from
                           * the FP32 rounding. Fused form, every element type; on curved hexahedra
                           * and with surface-flux anti-aliasing the mass equation takes the FP32 flux
                           * path instead of the float-float one (their metric or face quadrature
                           * takes rho v out of the solution space); ignored in FP64. */
    int surface_aa;       /* 1: surface-flux anti-aliasing as well (Sec. 2.2.1: the interface flux points
                           * are replaced by the m x m Gauss-Legendre points of each face, m = nq1d; the
                           * common flux is evaluated there and lifted through the face L2 projection).
                           * Single-instance hexahedral meshes, fused form (FP64, FP32, the low-Mach
                           * form). 0: flux points are the n x n solution-point traces. */
} fr_params;

/* Host description of one mesh instance (copied by fr_mesh_create). */
typedef struct {
    int n_hex;            /* number of hexahedra */
    int n_pri;            /* number of prisms */
    int n_verts;          /* number of vertices */
    const double *verts;  /* [n_verts][3] coordinates */
    const int *hex_v;     /* [n_hex][8] vertex ids, tensor order */
    const int *pri_v;     /* [n_pri][6] vertex ids */
    double period[3];     /* periodic box lengths; 0 = not periodic. Faces are matched modulo period */
    int n_tet;            /* number of tetrahedra (p = 3, flux anti-aliasing, fused form) */
    const int *tet_v;     /* [n_tet][4] vertex ids */
    int n_pyr;            /* number of pyramids (p = 3, flux anti-aliasing, fused form) */
    const int *pyr_v;     /* [n_pyr][5] vertex ids: base corners in tensor order, then the apex */
} fr_mesh_desc;

typedef struct fr_mesh fr_mesh;

/* Builds the operators, metrics and interface pairs of n_inst independent instances (one
 * fr_params each) and uploads them to the current CUDA device. Interfaces are found by matching
 * flux-point coordinates (modulo the periods); every face must find exactly one partner. The L side
 * of a pair is the element with the smaller global index; a self-pair takes the smaller local face
 * number as L. Returns FR_EMESH, FR_EUNSUPPORTED, FR_EINVAL or FR_ENOMEM on failure (*out = NULL). */
fr_status fr_mesh_create(const fr_mesh_desc *const *inst, int n_inst, const fr_params *prm, fr_mesh **out);

/* Frees every device and host resource of the handle. NULL is accepted. */
fr_status fr_destroy(fr_mesh *m);

/* Selects the kernel form used by later RHS and RK4 calls (fr_form). */
fr_status fr_set_form(fr_mesh *m, int form);

/* R = R(U): one RHS evaluation. U_dev and R_dev are device arrays of fr_num_values() elements in
 * the boundary layout and precision (double for FR_FP64, float otherwise); they must not overlap. */
fr_status fr_rhs(fr_mesh *m, const void *U_dev, void *R_dev, void *stream);

/* Same as fr_rhs with host arrays: copies U host->device, evaluates, copies R device->host and
 * synchronises the stream before returning. Host buffers may be pageable or pinned. */
fr_status fr_rhs_host(fr_mesh *m, const void *U_host, void *R_host, void *stream);

/* nsteps classical RK4 steps of size dt, in place, on the FP64 master state U_dev (double, device,
 * boundary layout). FR_FP64: stage states and the Runge-Kutta sum in FP64. Reduced precisions: the
 * stage states fl32(U) + c dt k and the Runge-Kutta sum are formed in FP32 (they are FP32 RHS inputs
 * and values either way), and the increment dt sum b_s k_s is added to U in FP64. */
fr_status fr_rk4_step(fr_mesh *m, void *U_dev, double dt, int nsteps, void *stream);

/* As fr_rk4_step on a host FP64 state: copies U host->device, advances nsteps, copies it back and
 * synchronises the stream. */
fr_status fr_rk4_step_host(fr_mesh *m, void *U_host, double dt, int nsteps, void *stream);

/* Autotuner: times every launch shape of the volume kernel of each hexahedral group (one element
 * type and order) on the given device state U_dev (R_dev is scratch output) and keeps the fastest
 * for later calls. Shapes: 0, 1, 2 = one element per CTA of 64, 128 or 256 threads; for FP32 (and
 * the mixed forms without hexahedral tensor cores) at p = 3 with flux anti-aliasing on affine
 * elements also 3, 4 = eight elements per CTA of 160 threads, each sum-factorised operator applied
 * to a whole field by one thread from registers (one CTA per SM with up to 255 registers, or two).
 * chosen[i] (n_chosen entries, may be NULL) receives the shape index of group i. Where the groups can
 * share one launch per phase (fr_set_merged), it also times a whole RHS both ways and keeps the faster
 * (fr_mesh_info reports the launches per RHS). Shapes 0, 1 and 2
 * evaluate each output with the same operations (results do not depend on the choice among them);
 * shapes 3 and 4 sum the projection's 1D factors in another order (the factors commute), so FP32
 * results then differ at the FP32 rounding level. Synchronises the stream. */
fr_status fr_autotune(fr_mesh *m, const void *U_dev, void *R_dev, int *chosen, int n_chosen, void *stream);

/* Kernel groups (blocks of one element type and order, launched together): info[0..5] of group
 * `group` = element type (0 hex, 1 prism, 2 tetrahedron, 3 pyramid), order p, quadrature points per
 * line, elements, current volume-kernel shape, number of shapes it can run. FR_EINVAL past the last
 * group. fr_set_group_shape sets one hexahedral group's shape (e.g. a choice of fr_autotune kept from
 * an earlier run); FR_EUNSUPPORTED for a shape the group cannot run. */
fr_status fr_group_info(const fr_mesh *m, int group, long long *info);
fr_status fr_set_group_shape(fr_mesh *m, int group, int shape);

/* on = 1: one launch per phase over all the handle's element groups (hexahedra p = 3 and 4 and prisms,
 * flux anti-aliasing on the CUDA cores, affine elements, 2 to 4 groups; else FR_EUNSUPPORTED): three
 * launches per RHS whatever the number of instances, element types and orders, each CTA taking its
 * share of every group in turn. The kernel's registers and shared memory are those of its largest
 * group, so it can run fewer CTAs per SM than the per-group launches (on = 0, the default);
 * fr_autotune times both on the caller's state and keeps the faster. Results are bit for bit those of
 * the per-group launches, except on FP64 hexahedral-only handles, whose per-group launches evaluate
 * each interface pair once with the L side's normal while the merged launch evaluates each side with
 * its own: where the two normals are negatives only to the last bit (sheared meshes) the results agree
 * to rounding. Recaptures the RK4 graph. */
fr_status fr_set_merged(fr_mesh *m, int on);

/* Reduced precisions (FP32 and the mixed forms): on = 1 forms the RK4 stage states
 * u_{s+1} = U + c_{s+1} dt k_s and the Runge-Kutta sum sum_s b_s k_s in FP64 from the FP64 master
 * state (Sec. 3's RK4 with only the RHS evaluations in the reduced precision); on = 0, the default,
 * forms both in FP32 from fl32(U) and keeps FP64 for the update of U at the end of the step, which
 * moves about half the bytes per stage. No effect on FP64 handles. Takes effect from the next step
 * (switch between steps, not between the stages of one); recaptures the RK4 graph. */
fr_status fr_set_rk_fp64_stages(fr_mesh *m, int on);

/* Sets the volume-kernel launch shape (0..5, as for fr_autotune) of every hexahedral group;
 * FR_EUNSUPPORTED if a group cannot run it. Takes effect at the next launch (recaptures the RK4 graph). */
fr_status fr_set_volume_shape(fr_mesh *m, int shape);

/* Blocks until the stream's work on this handle has finished and returns the latched device
 * status (FR_OK or FR_ENONPHYS), clearing it. */
fr_status fr_sync_status(fr_mesh *m, void *stream);

/* Counts: info[0] elements, info[1] values of U (= DOF), info[2] flux points, info[3] interface
 * pairs, info[4] instances, info[5] kernel launches per RHS in the current form,
 * info[6] bytes of device memory owned by the handle. */
fr_status fr_mesh_info(const fr_mesh *m, long long *info);

/* Number of values of U (elements x 5 x points, summed over instances and element types). */
long long fr_num_values(const fr_mesh *m);

/* Physical coordinates of every solution point, [point in boundary order][3], into a host array
 * of fr_num_values()/5*3 doubles. */
fr_status fr_sol_coords(const fr_mesh *m, double *xyz_host);

/* Per-instance value offsets: off[i] is the first value of instance i in U, off[n_inst] the total. */
fr_status fr_instance_offsets(const fr_mesh *m, long long *off);

/* Diagnostics of a device state U (and RHS R, may be NULL), per instance i, into the host array
 * out[i*8 + k]: k=0 volume sum W detJ, 1 E_k = <rho|v|^2/2>, 2 eps = -dE_k/dt from R, 3..7 the
 * quadrature-weighted sums of R per variable. W are the solution-point quadrature weights.
 * Synchronises the stream. */
fr_status fr_diagnostics(fr_mesh *m, const void *U_dev, const void *R_dev, double *out, void *stream);

/* Same results as fr_diagnostics, for callers that must not allocate device memory (for example
 * while another framework owns the device memory budget, in a real-time loop that cannot afford the
 * device-wide synchronisation a cudaMalloc may cause, or while a thread captures other work into a
 * CUDA graph in global mode, where cudaMalloc is not allowed). The paper has no counterpart: this is
 * a service of the library. It allocates nothing: its accumulators are a fixed array of
 * 1024 x 8 doubles (64 KiB) compiled into the library, which every GPU that loads the library holds
 * until the process exits; handles with more than 1024 instances get FR_EINVAL. fr_mesh_create looks
 * up that array's device address (with the handle's device current), so this call does no set-up of
 * its own; the handle's device must be the current device (else FR_EINVAL). All calls share the one
 * array and each call clears only the slots it uses: calls that overlap on the GPU (other streams,
 * other threads) race and give wrong sums. While another thread captures a stream in global mode,
 * pass a non-blocking stream: work on the legacy default stream (NULL) would join that capture's
 * stream and invalidate it. An instance without elements reports 0 for E_k and eps. Synchronises
 * the stream. */
fr_status fr_diagnostics_noalloc(fr_mesh *m, const void *U_dev, const void *R_dev, double *out, void *stream);

/* Copies an intermediate array of the last UNFUSED RHS to a host FP64 array, for stage-level
 * checks. which: 0 U^(f) [var][fpt], 1 C^(f) [var][fpt], 2 physical gradient Q^(u)
 * [elem][var][dim][pt], 3 Q^(f) [var][dim][fpt], 4 projected flux F~^(u) [elem][var][dim][pt],
 * 5 D^(f) [var][fpt]. Flux points use the global order elem-major, local face order above.
 * n_host is the capacity in doubles; the needed size is returned in *n_needed. Synchronises. */
fr_status fr_stage(fr_mesh *m, int which, double *host, long long n_host, long long *n_needed);

/* Debug flags: bit 0 keeps a copy of the unfused form's physical gradient Q^(u) for fr_stage(2).
 * Bit 1 makes the first bounded device wait of every CTA give up at once (the tensor-core completion
 * wait of the mixed forms' volume kernels and the hexahedral state prefetch of p = 3): the kernel
 * reports it (FR_ETIMEOUT at the next fr_sync_status or call), waits for its own asynchronous work
 * with the normal bound, releases its tensor memory and returns (the tensor-core kernels leave their
 * remaining elements unevaluated; the prefetch falls back to a global-memory read, so R stays
 * correct). It exercises the failure path without any fault. */
fr_status fr_set_debug(fr_mesh *m, int flags);

/* RK4 CUDA graphs (on = 1, the default): fr_rk4_step captures one step (stage states, RHS launches,
 * stage updates) into a graph on first use and replays it once per step; it recaptures when the
 * state pointer, dt, stream or kernel form changes. The legacy default stream and per-kernel timing
 * use plain launches. */
fr_status fr_set_graph(fr_mesh *m, int on);

/* Mixed forms only: on = 1 also moves the x-y factor of the hexahedral interpolation and
 * projection (the dense Kronecker blocks B (x) B and Pj (x) Pj of the Sec. 4 factorisation) to the
 * split-product tensor-core path used for the prisms. Default 0: the hexahedra keep the FP32 1D
 * sweeps on the CUDA cores, which are faster on GB300 (the dense block costs more multiply-adds and
 * shared memory than the sweeps save). Results then differ from FR_FP32 at the split-product
 * rounding only. Takes effect at the next launch (and recaptures the RK4 graph). */
fr_status fr_set_hex_tensor_cores(fr_mesh *m, int on);

/* Mixed forms only: on = 1 moves the interpolation of the 20 fields (state and corrected gradient)
 * to the 125 quadrature points of every tetrahedron and pyramid (a dense 125 x NU operator, Sec. 1
 * element types without the Sec. 4 factorisation) to the split-product tensor-core path: one
 * M = 128 (quadrature points) x N = 32 (fields) MMA chain per element over K = 3 NU, the operator
 * split once per CTA. Default 0: the volume kernel of these types is bound by latency, and the
 * tensor-core tiles add shared memory and a wait per element, so the FP32 products
 * on the CUDA cores are faster on GB300 (volume kernel 1.24 vs 1.47 ms per launch on the 24^3
 * Kuhn box in the low-Mach form). Results
 * then differ from FR_FP32 at the split-product rounding only. Takes effect at the next launch (and
 * recaptures the RK4 graph). */
fr_status fr_set_dense_tensor_cores(fr_mesh *m, int on);

/* Per-kernel timing (on = 1): CUDA events are recorded on the launching stream around every later
 * launch. fr_kernel_times waits for them and returns, per kernel id, the summed milliseconds and the
 * launch count, then clears the record. Ids: 0, 1, 2 fused phases (face solution, volume group,
 * interface group); 10 + k unfused kernel k = 1..13 in the paper's order; 30 RK4 stage update.
 * Arrays have n_ids entries. */
fr_status fr_set_timing(fr_mesh *m, int on);
fr_status fr_kernel_times(fr_mesh *m, double *ms, long long *count, int n_ids);

/* ---------------------------------------------------------------------------------------------
 * Partitioned single mesh (one part per GPU). The RHS needs neighbour data at two points only, the
 * boundaries of the paper's kernel groups (Sec. 2.2, kernel-grouping figure): the face solution
 * U^(f) before con_u, and the face data of comm_flux before it. A single-instance mesh is split
 * into nparts contiguous ranges of its global element order (part r owns elements
 * [floor(ne r / nparts), floor(ne (r+1) / nparts))); each part holds its own elements and flux
 * points plus one halo slot per remote partner point. An RHS on part r is
 *     fr_rhs_phase(0); fr_halo_pack(0) -> exchange -> fr_halo_unpack(0);
 *     fr_rhs_phase(1); fr_halo_pack(1) -> exchange -> fr_halo_unpack(1);
 *     fr_rhs_phase(2)
 * where "exchange" sends the segment of peer q of the send buffer to q and receives q's segment
 * into the same place of the receive buffer (any transport: NCCL, MPI, or device copies). Each side
 * of a pair evaluates its own point's common flux with the pair's global L/R roles, so the parts'
 * R concatenated equal the single-handle RHS bit for bit. RK4 steps go the same way through
 * fr_rk4_stage. Surface-flux anti-aliasing, the unfused form, fr_rhs and fr_rk4_step are
 * FR_EUNSUPPORTED on a part of a mesh with nparts > 1.
 * ------------------------------------------------------------------------------------------- */

/* Exchange plan of part `part` of nparts, computed on the host only (no device is touched).
 * info[0..5]: first and one-past-last own global element, own flux points, halo points, elements
 * and flux points of the whole mesh. counts[q] (nparts entries, may be NULL): points exchanged with
 * peer q (the same number in both directions). send_g / recv_g (cap entries each, may be NULL):
 * whole-mesh flux-point indices (element-major, local face order) of the points this part sends and
 * of the remote points it receives, in buffer order. */
fr_status fr_partition_plan(const fr_mesh_desc *desc, const fr_params *prm, int nparts, int part,
                            long long *info, long long *counts, long long *send_g, long long *recv_g,
                            long long cap);

/* Builds part `part` of nparts of a single-instance mesh on the current device (see above); U and R
 * of the handle hold the own elements only, in the boundary layout. */
fr_status fr_mesh_create_part(const fr_mesh_desc *desc, const fr_params *prm, int nparts, int part, fr_mesh **out);

/* info[0..6]: nparts, part, first and one-past-last own global element, halo points, values per
 * point of exchange 0 (5: the face solution) and of exchange 1 (4: the own-normal viscous flux, or
 * 6 in the low-Mach FP32 form: plus the float-float mass flux as two floats). counts[q] (nparts
 * entries, may be NULL): points exchanged with peer q. */
fr_status fr_halo_info(const fr_mesh *m, long long *info, long long *counts);

/* Packs (after fr_rhs_phase(what)) this part's face data that its peers need into the device buffer
 * send_dev, or unpacks the peers' data from recv_dev into the halo slots (before fr_rhs_phase(what +
 * 1)). Buffers hold, peer by peer in increasing rank order, nvar x counts[q] values of the compute
 * precision (double for FR_FP64, float otherwise), var-major. Asynchronous on `stream`. */
fr_status fr_halo_pack(fr_mesh *m, int what, void *send_dev, void *stream);
fr_status fr_halo_unpack(fr_mesh *m, int what, const void *recv_dev, void *stream);

/* One phase of the fused RHS: 0 face solution (disu), 1 volume group (con_u .. tdivtpcorf, writes
 * R~ into R), 2 interface group (comm_flux, tdivtconf, negdivconf: finishes R). Same arguments as
 * fr_rhs; phases 0, 1, 2 in order on one stream are one fr_rhs. */
fr_status fr_rhs_phase(fr_mesh *m, int phase, const void *U_dev, void *R_dev, void *stream);

/* One phase (0, 1, 2 as for fr_rhs_phase) of stage `stage` (0..3) of a classical RK4 step on the
 * FP64 master state U_dev, with the stage update after phase 2 (as fr_rk4_step does it); stages 0..3
 * with phases 0, 1, 2 each, in order, are one fr_rk4_step(nsteps = 1). The stage states and the
 * Runge-Kutta sum live in the handle. On a part of a partitioned mesh the halo exchanges go between
 * the phases, as for an RHS. Fused form; asynchronous on `stream`. */
fr_status fr_rk4_stage(fr_mesh *m, int stage, int phase, void *U_dev, double dt, void *stream);

/* Text of the last error on the calling thread ("" if none). */
const char *fr_last_error(void);

/* Measures the device's sustained FMA throughput: out[0] FP64 GFLOP/s, out[1] FP32 GFLOP/s
 * (CUDA-core FMA chains over every SM, timed with events). Synchronises. */
fr_status fr_probe_fma(double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FR_GB300_H */
