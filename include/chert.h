/*
 * chert.h -- C ABI of libchert.so, the sm_103a implementation of the hot path of
 * CHERT (Darwis et al., "CHERT: Cached Hamiltonian-Enhanced Ray Tracing in
 * Viscoelastic Anisotropic Media"): the directional cache build and the
 * cache-lookup shortest-path traveltime relaxation.
 *
 * Conventions shared by every entry point
 *   - Every function returns a status code (CHERT_OK = 0 or a negative error)
 *     and never aborts; chert_last_error() gives a message for the calling thread.
 *   - "device" pointers are CUDA device memory of the current device; the caller
 *     owns every buffer.  The library allocates no device memory: where it needs
 *     scratch, the caller passes a workspace whose size a *_workspace_bytes()
 *     query returns.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is only
 *     enqueued unless a function says it synchronises.
 *   - Units are SI: moduli in (m/s)^2 (density normalised), lengths in m,
 *     traveltimes in s, angles in rad.
 *   - Floating-point buffers are double for CHERT_FP64 and float for
 *     CHERT_FP32 / CHERT_MIXED; with CHERT_FP32_ACC64 (3D traveltimes) the
 *     cache is float and tauR/tauI are double.
 *   - 2D lattice: node = x + nx*z (z = depth).  3D: node = x + nx*(y + ny*z).
 */
#ifndef CHERT_H
#define CHERT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define CHERT_OK        0
#define CHERT_EINVAL   -1   /* bad argument (message in chert_last_error)      */
#define CHERT_ENOMEM   -2   /* workspace smaller than *_workspace_bytes()      */
#define CHERT_ECUDA    -3   /* a CUDA runtime call failed                       */
#define CHERT_ETIMEOUT -4   /* relaxation hit its cycle cap before converging  */

/* ---- wave modes, kernels, precisions ------------------------------------ */
#define CHERT_QP  0
#define CHERT_QSV 1
#define CHERT_QSH 2

#define CHERT_OEV 0         /* g-Hamiltonian, Eq. 12                           */
#define CHERT_MEV 1         /* g*-Hamiltonian, Eq. 13-14                       */

#define CHERT_FP64  0       /* every step in double                            */
#define CHERT_FP32  1       /* every step in float                             */
#define CHERT_MIXED 2       /* float scan, float-float (~48-bit) root polish and
                               ray quantities, float storage and relaxation    */
#define CHERT_FP32_ACC64 3  /* chert_traveltime on 3D lattices only: float
                               cache and edge weights, traveltimes accumulated
                               in float-float (~48-bit) and returned as double */

/* One cache class k (a layer, facies, cell or tilt group).  Eq. 2:
 * a = aR - i*aI per Voigt component (a11, a13, a33, a44, a66) of a VTI solid
 * whose symmetry axis is tilted by (tilt, azim) = (theta_0, phi_0), Eq. 35. */
typedef struct {
    double aR[5];
    double aI[5];
    double rho;      /* stored only, Eq. 26 */
    double tilt;     /* theta_0 */
    double azim;     /* phi_0 (3D; 0 in 2D) */
} chert_class;

/* Thomsen (Vp0, Vs0, eps, delta, gamma) and quality factors to one class:
 * a33 = Vp0^2, a44 = Vs0^2, a11 = a33(1+2 eps), a66 = a44(1+2 gamma),
 * a13 = sqrt((a33-a44)(a33(1+2 delta)-a44)) - a44, and (Eq. 2 with the
 * per-component reading of the paper's Table 2) aI = aR/Q with
 * Q11 = Q13 = Q33 = qp, Q44 = Q66 = qs.  Host only.
 * Errors: CHERT_EINVAL if out is NULL, a velocity or Q is not positive, or
 * delta leaves no real a13. */
int chert_thomsen_to_class(double vp0, double vs0, double eps, double delta,
                           double gamma, double qp, double qs, double rho,
                           double tilt, double azim, chert_class* out);

/* Eq. 2 for a medium given as real moduli aR = (a11, a13, a33, a44, a66) and
 * one quality factor per component q[5] (the paper's Table 2 lists both):
 * aI[i] = aR[i] / q[i], and 0 where q[i] is +inf (elastic).  Host arrays of
 * 5 doubles.  Host only.
 * Errors: CHERT_EINVAL if a pointer is NULL, a q[i] is not positive, or
 * a33 or a44 is not positive. */
int chert_moduli_to_class(const double* aR, const double* q, double rho,
                          double tilt, double azim, chert_class* out);

/* chert_thomsen_to_class for n classes (host arrays of length n; out holds
 * n records).  Stops at the first invalid class (CHERT_EINVAL, index in the
 * message). */
int chert_thomsen_to_classes(int64_t n, const double* vp0, const double* vs0,
                             const double* eps, const double* delta, const double* gamma,
                             const double* qp, const double* qs, const double* rho,
                             const double* tilt, const double* azim, chert_class* out);

/* ---- cache build (Eq. 4-14, 26, 35-36) ---------------------------------- */

/* Output arrays of the directional cache C(m, k, theta), all device, each laid
 * out [n_modes][n_classes][n_dir] with n_dir = 4*M (Eq. 26, Table 1).
 * Directions d index the slowness angle theta_d = d*(pi/2)/M of the class's
 * local symmetry-axis frame; the stored values are global:
 *   V, A, Q     ray velocity (m/s), ray attenuation (s/m), ray quality (Eq. 11)
 *   rx, rz      unit ray direction r in the global x-z plane (Eq. 36)
 *   theta       global real slowness angle theta_d + tilt, from +z toward +x
 *   vartheta    the imaginary slowness angle of the homogeneous solution, signed
 *               as seen from direction d (Eq. 9)
 *   flag        0 = valid, 1 = no acceptable (decaying) root; V, A, Q, rx, rz,
 *               vartheta are NaN then and the lookup skips the entry.
 *   ry, phi     3D caches only (chert_build_cache_3d): the y component of r and
 *               the global slowness azimuth; theta is then the global polar
 *               angle.  2D builds neither read nor write them (may be NULL).
 * Any pointer except flag, V and rx/rz (and ry in 3D) may be NULL to skip
 * that output. */
typedef struct {
    void*    V;
    void*    A;
    void*    Q;
    void*    rx;
    void*    rz;
    void*    theta;
    void*    vartheta;
    uint8_t* flag;
    void*    ry;
    void*    phi;
} chert_cache_arrays;

/* Homogeneity search settings.  The roots of the residual
 * f(vartheta) = (v^R x v^I)_y / |v^R|^2 (Eq. 9) are the sign changes of f on
 * the grid vartheta_k = k*scan_step, |k| <= scan_half, plus exact zeros on the
 * grid; each is polished to a bracket below 1e-14 rad (FP64, MIXED) or to
 * float resolution (FP32).  The chosen root is the decaying one (v_I <= 1e-9
 * v_R, stored A clamped at 0) of least |vartheta|, the negative one on a tie.
 * Defaults used by the paper's [-30, 30] deg bracket: scan_step = 0.001 deg,
 * scan_half = 30000. */
typedef struct {
    int    M;            /* slowness angles per quadrant, >= 1 (1 deg: M = 90) */
    double scan_step;    /* rad, > 0 */
    int    scan_half;    /* >= 1 */
    int    kernel;       /* CHERT_OEV or CHERT_MEV */
    int    precision;    /* CHERT_FP64, CHERT_FP32 or CHERT_MIXED */
} chert_cache_params;

/* Build the cache for n_classes classes (device array d_classes) and n_modes
 * wave modes (host array `modes`, values CHERT_QP/QSV/QSH, distinct, <= 3).
 * One warp solves each distinct folded angle (0..90 deg) of each (mode,
 * class) and writes the up to four mirrored entries.  Errors: CHERT_EINVAL
 * (counts, params, NULL outputs), CHERT_ECUDA. */
int chert_build_cache(const chert_class* d_classes, int n_classes,
                      const int* modes, int n_modes,
                      const chert_cache_params* params,
                      const chert_cache_arrays* out, void* stream);

/* Solve only the listed solves of a cache (same arguments and arrays as
 * chert_build_cache), leaving the other entries untouched.  A solve is the
 * folded angle j of class k in mode slot m, numbered
 * m*n_classes*(M+1) + k*(M+1) + j (device int64 list), and writes its up to
 * four mirrored entries.  Used to recompute the entries a surrogate cache
 * marks as needing the exact solver. */
int chert_build_cache_items(const chert_class* d_classes, int n_classes,
                            const int* modes, int n_modes,
                            const chert_cache_params* params,
                            const int64_t* d_items, int64_t n_items,
                            const chert_cache_arrays* out, void* stream);

/* Threads per CTA of the cache build's finish pass (the solves with no
 * decaying root within 2,048 grid points per side), process-wide: 0 (default)
 * 1024 for builds of at most 65,536 solves and 256 above; or 256, 512, 1024.
 * The cache is the same for every choice (the nearest 64-point slice with a
 * root wins); this is for measurement and tuning.  Returns the previous
 * setting, or CHERT_EINVAL. */
int chert_set_cache_finish_threads(int threads);

/* 3D cache (Eq. 35, the 3D TTI extension of the paper's experiments): entry
 * d = i*n_az + j of class k is the global slowness direction of polar angle
 * (i + 1/2)*pi/n_pol and azimuth j*2*pi/n_az (arrays [n_modes][n_classes]
 * [n_az*n_pol]).  Each direction is expressed in the class's symmetry-axis
 * frame (e_x', e_y', e_z') given by its tilt theta0 and azimuth phi0; the
 * medium being rotationally symmetric about e_z', the homogeneity search runs
 * in the sagittal plane at the local polar angle folded into [0, pi/2], and
 * the ray is turned to the local azimuth, mirrored back and written in the
 * global frame (rx, ry, rz).  Same search settings and root rule as
 * chert_build_cache (params->M is ignored); one solve per entry.  Errors:
 * CHERT_EINVAL (also for a NULL ry), CHERT_ECUDA. */
int chert_build_cache_3d(const chert_class* d_classes, int n_classes, const int* modes, int n_modes,
                         int n_az, int n_pol, const chert_cache_params* params,
                         const chert_cache_arrays* out, void* stream);

/* ---- direction lookup (Eq. 27-28) --------------------------------------- */

/* For every (mode, class, stencil offset o): the cache entry whose ray
 * direction r has the largest dot product with d = o/|o| (both float64 for
 * CHERT_FP64, float32 otherwise; products rounded separately, ties to the
 * lower entry index, flagged entries skipped; the dot product is summed as
 * ((dx*rx) + (dy*ry)) + (dz*rz), the middle term only when the cache has ry).
 * Writes device arrays
 * [n_modes][n_classes][n_off]: idx (int32, -1 if a class has no valid
 * entry), Vsel and Asel (the entry's V and A, NaN for idx = -1).
 * offsets: host int32 [n_off][3] = (ox, oy, oz), 1 <= n_off <= 512, oy = 0
 * in 2D.  Errors: CHERT_EINVAL, CHERT_ECUDA. */
int chert_edge_table(const chert_cache_arrays* cache, int n_modes, int n_classes,
                     int n_dir, int precision, const int32_t* offsets, int n_off,
                     int32_t* d_idx, void* d_Vsel, void* d_Asel, void* stream);

/* Nodewise angular coverage of a 2D cache (the paper's angular-coverage
 * validation; it names coverage ratio, missing-angle ratio and branch
 * mismatch without formulas -- this is one reading).  For every (mode, class)
 * k and stencil direction d = o/|o|:
 *   covered     two cyclically adjacent valid entries e, e+1 whose ray
 *               directions are less than 90 deg apart hold d on the closed
 *               short arc between them (a bracket);
 *   mismatched  d is covered, and the entry of chert_edge_table's lookup is
 *               neither end of the first-arrival bracket: the bracket with the
 *               largest ray velocity interpolated at d, V_e + t (V_e+1 - V_e)
 *               with t = cross(r_e, d) / cross(r_e, r_e+1), ties to the lower
 *               e (at a qSV fold, the path search would take a slower branch).
 * and, with a reference cache's flags (d_truth_flag, same layout; may be
 * NULL), missing = entries valid in the reference but flagged here.
 * Bracket arithmetic in double, each operation rounded separately; the
 * lookup in the cache's precision as chert_edge_table.  cache: rx, rz, V,
 * flag of [n_modes][n_classes][n_dir] (n_dir = 4M).  offsets: host int32
 * [n_off][3], oy = 0, 1 <= n_off <= 512.  Outputs: device int32
 * [n_modes][n_classes] each (covered and mismatched count directions, out of
 * n_off; missing counts entries, out of n_dir).
 * Errors: CHERT_EINVAL (NULL, counts, 3D offsets), CHERT_ECUDA. */
int chert_angular_coverage(const chert_cache_arrays* cache, int n_modes, int n_classes, int n_dir,
                           int precision, const int32_t* offsets, int n_off,
                           const uint8_t* d_truth_flag, int32_t* d_covered, int32_t* d_mismatched,
                           int32_t* d_missing, void* stream);

/* ---- traveltime relaxation (Eq. 22, 27-33) ------------------------------ */

/* Scratch bytes chert_traveltime needs for this problem size (the class
 * tables only; enough for every lattice). */
size_t chert_traveltime_workspace_bytes(int n_modes, int n_classes, int n_off,
                                        int precision, int n_sources);

/* Scratch bytes for this problem on an nx x ny x nz lattice, including (2D,
 * ny = 1) the per-node weight area: with the standard secondary-node stencil and too
 * many classes for the class-pair table in shared memory (e.g. one class per
 * node), chert_traveltime precomputes each node's directed edge weights in row-
 * and column-major layouts, n_modes x 2 x n_off x nodes values each, when the
 * workspace it is given holds them, and otherwise relaxes with weights read
 * through the class map (same results, slower).  Returns 0 for invalid
 * counts. */
size_t chert_traveltime_workspace_bytes_grid(int n_modes, int n_classes, int n_off, int precision,
                                             int n_sources, int nx, int ny, int nz);

/* Propagation and attenuation traveltime fields for every (source, mode) of
 * a cache, on a lattice nx x ny x nz with spacing dx: 2D with ny = 1 (cache
 * from chert_build_cache; offsets with oy = 0), 3D with ny > 1 (cache from
 * chert_build_cache_3d, whose ry the lookup uses).  Node index
 * x + nx*(y + ny*z).
 *   d_class_of_node  device int32 [nz*ny*nx], values in [0, n_classes)
 *   offsets          host int32 [n_off][3], a set closed under negation
 *   sources          host int64 [n_sources] node indices
 * Each directed edge i -> j = i + o costs, with the selected (V, A) of the
 * end classes (Eq. 28-30), wR = L/(0.5 (V_ki + V_kj)) and wI = L*0.5(A_ki + A_kj),
 * L = dx|o|.  tauR and tauI are the fixed points of Eq. 31 from tau(source) = 0,
 * solved separately; parR/parI (may be NULL) follow the rule
 * par_j = argmin_i (tau_i + w_ij), ties to the smallest i, par(source) =
 * source, par = -1 and tau = +inf where unreachable (Eq. 33).
 * Outputs are device arrays [n_sources][n_modes][nz*ny*nx].
 * 2D cycles sweep lines (rows and columns, both ways); 3D cycles sweep planes
 * of constant z, y and x, both ways.  Which 2D scheduler runs (sweeps, the
 * paper's block-heap marching, or the default hybrid of the two) is set by
 * chert_set_relax_scheduler; all give the same fields and parents.
 * max_cycles caps the sweep cycles per field (under block-heap marching: the
 * verification passes, and max_cycles x blocks x 8 block relaxations); a
 * field that has not converged after it returns CHERT_ETIMEOUT (its values
 * are valid upper bounds; the nodes that a block-heap field cut off mid-way
 * has not reached hold +inf).
 * Synchronises on `stream` once at the end to read the convergence status.
 * Errors: CHERT_EINVAL, CHERT_ENOMEM (workspace too small), CHERT_ECUDA,
 * CHERT_ETIMEOUT. */
int chert_traveltime(const chert_cache_arrays* cache, int n_modes, int n_classes,
                     int n_dir, int nx, int ny, int nz, double dx,
                     const int32_t* d_class_of_node, const int32_t* offsets,
                     int n_off, const int64_t* sources, int n_sources,
                     int precision, int max_cycles,
                     void* d_tauR, void* d_tauI, int32_t* d_parR, int32_t* d_parI,
                     void* d_workspace, size_t workspace_bytes, void* stream);

/* Launch shape of the 2D relaxation specialised to the standard stencil:
 * nodes of a line per thread (1, 2 or 4; threads = line length / ppt,
 * rounded up to a warp, at most 512).  0 (the default) chooses from the line
 * length; a forced value applies wherever the line fits.  Process-wide (for
 * an autotuner that times each choice on its problem).  Returns the previous
 * setting, or CHERT_EINVAL for other values.  Results do not depend on it. */
int chert_set_relax_points_per_thread(int ppt);

/* Scheduler of the 2D relaxation, process-wide:
 *   0 ordered sweep cycles;
 *   1 the paper's block-heap marching (Eq. 32): 32 x 32 node blocks keyed by
 *     the least traveltime that may still propagate from them, the smallest
 *     taken next and relaxed inside to local convergence (staged with a halo
 *     of the stencil's reach in shared memory), the neighbours within reach
 *     of a changed node re-keyed;
 *   2 (default) hybrid: at most 6 sweep cycles, then block-heap marching, from the
 *     source, for the fields that have not converged (one more launch,
 *     whose CTAs of converged fields return at once);
 *   3 frontier label correcting: one CTA per field component; the nodes
 *     whose traveltime fell in a round push tau_i + w_ij to their
 *     out-neighbours with an unsigned atomicMin on the traveltimes' bit
 *     patterns (non-negative values order like their bits) and mark the
 *     ones they lowered for the next round; a pull pass then writes the
 *     parents.  Needs the class-pair table and two frontier bitmaps (one bit
 *     per node) in shared memory, else CHERT_EINVAL; max_cycles x max(nx, nz)
 *     rounds at most.
 * All return the same fixed point of Eq. 31 and the same parents; they
 * differ in the work done.  Under scheduler 1, a 2D chert_traveltime whose
 * stencil reaches more than 8 nodes returns CHERT_EINVAL; under 2 it sweeps
 * only, as it does when max_cycles <= 6.  3D lattices always sweep.
 * scheduler < 0 queries without changing.  Returns the previous (or current)
 * setting, or CHERT_EINVAL for scheduler > 3. */
int chert_set_relax_scheduler(int scheduler);

/* The same relaxation as chert_traveltime, enqueued on `stream` without any
 * host synchronisation or host-to-device copy: sources are a device int64
 * array, the offsets travel by value to the kernels, and the convergence
 * status lands in d_status (device int32[2]): [0] the first index
 * field*2 + component (field = source*n_modes + mode) that hit max_cycles, or
 * -1; [1] 1 if the class map held ids outside [0, n_classes), else 0.  A
 * source outside the lattice yields an all-unreachable field.  Repeated
 * problems (many sources and modes, several models) can so be recorded once
 * as a CUDA graph and replayed as one launch.  Errors (host-side argument
 * checks): CHERT_EINVAL, CHERT_ENOMEM (workspace too small), CHERT_ECUDA. */
int chert_traveltime_enqueue(const chert_cache_arrays* cache, int n_modes, int n_classes, int n_dir,
                             int nx, int ny, int nz, double dx, const int32_t* d_class_of_node,
                             const int32_t* offsets, int n_off, const int64_t* d_sources, int n_sources,
                             int precision, int max_cycles, void* d_tauR, void* d_tauI, int32_t* d_parR,
                             int32_t* d_parI, void* d_workspace, size_t workspace_bytes, int32_t* d_status,
                             void* stream);

/* 3D tile shape of the plane sweeps, process-wide: 0 (default) 32 x 16 nodes
 * per tile, 1 64 x 8 (longer contiguous rows along x, more halo).  For an
 * autotuner; the fields and parents do not depend on it.  Returns the
 * previous setting, or CHERT_EINVAL. */
int chert_set_relax3d_tile(int tile);

/* One lattice of chert_traveltime_batch: chert_traveltime_enqueue's
 * arguments for it (its own cache, classes, class map, device sources,
 * outputs, workspace and device status int32[2]).  3D: ny > 1, workspace of
 * chert_traveltime_workspace_bytes.  2D: ny = 1, workspace of
 * chert_traveltime_workspace_bytes_grid (room for per-node weights). */
typedef struct {
    const chert_cache_arrays* cache;
    int n_classes, n_dir;
    int nx, ny, nz;
    double dx;
    const int32_t* d_class_of_node;
    const int64_t* d_sources;
    int n_sources;
    void* d_tauR;
    void* d_tauI;
    int32_t* d_parR;
    int32_t* d_parI;
    void* d_workspace;
    size_t workspace_bytes;
    int32_t* d_status;
} chert_lattice;

/* Several lattices of uneven size (up to 48; all 3D or all 2D; same modes,
 * precision, stencil and cycle cap) relaxed in persistent launches: every
 * lattice's field components are work items, numbered largest lattice first;
 * a grid of one wave of resident CTAs claims them from the device counter
 * d_counter (device uint64, zeroed here on `stream`) until none is left.
 *   3D: ONE launch of the plane-sweep kernel; each item relaxed as
 *       chert_traveltime relaxes it (same fields, parents and status, bit for
 *       bit).
 *   2D: the lattices the specialised sweep kernel takes with the radius-5
 *       stencil, grouped by launch shape (nodes a thread, class-pair table or
 *       per-node weights), each group one launch of up to 24 lattices,
 *       attenuation components first; each item relaxed as chert_traveltime
 *       relaxes it under the sweeps scheduler (scheduler 0: no block-heap
 *       continuation).  Other 2D lattices are relaxed on their own, as
 *       chert_traveltime_enqueue relaxes them.
 * Edge tables and class checks run per lattice before the launches.  No host
 * synchronisation: capturable.  Errors: as chert_traveltime_enqueue;
 * CHERT_EINVAL for a mix of 2D and 3D lattices. */
int chert_traveltime_batch(const chert_lattice* lattices, int n_lattices, int n_modes, int precision,
                           const int32_t* offsets, int n_off, int max_cycles,
                           unsigned long long* d_counter, void* stream);

/* ---- cache surrogate (a learned stand-in for the cache build; no counterpart in the paper)
 * One MLP per wave mode, 7 -> 256 -> 256 -> 256 -> 256 -> 5 with SiLU hidden
 * activations, BF16 operands, FP32 accumulation and FP32 master weights.  It
 * predicts the correction of a cache entry (the homogeneity solve of Eq. 9-11
 * at a folded slowness angle theta in [0, pi/2]) to the exact elastic ray
 * quantities of the same medium:
 *   inputs  x = (theta, Vs0/Vp0, eps, delta, gamma, 1/Qp, 1/Qs), each scaled to
 *           [-1, 1] over the training range (theta in [0, pi/2], Vs0/Vp0 in
 *           [0.49, 0.6], eps in [0.04, 0.31], delta in [-0.11, 0.21], gamma in
 *           [0, 0.21], 1/Q in [0.004, 0.051]); rows are padded to 8 floats;
 *   outputs (V/Vg - 1, log(A/A0), psi - psi_el, validity logit, vartheta),
 *           stored standardised (y = (raw - out_mean) / out_std; out_mean[3] = 0,
 *           out_std[3] = 1), with Vg, psi_el the elastic group velocity and ray
 *           angle of the real moduli and A0 the attenuation Im(1/c) of the
 *           homogeneous plane wave (complex phase velocity c of the complex
 *           Christoffel block along theta) projected on the elastic ray.  For
 *           qSH, whose homogeneous plane wave is the exact solution, the cache
 *           takes A0 itself and ignores output 1.
 * Parameter vector (float, chert_mlp_param_count() values): W0 [256 x 7], b0,
 * W1..W3 [256 x 256], b1..b3, W4 [5 x 256], b4, out_mean [5], out_std [5]
 * (W as [out][in]). */
size_t chert_mlp_param_count(void);
size_t chert_mlp_workspace_bytes(int64_t n, int training);

/* GEMMs with M >= 128 rows and N a multiple of 128 run on the tcgen05 tensor
 * cores (TMA-fed, accumulator in tensor memory), the others on a CUDA-core
 * kernel.  enable = 0 sends every GEMM to the CUDA-core kernel (process-wide;
 * used to compare the two).  Returns the previous setting. */
int chert_mlp_set_tensor_cores(int enable);

/* Every mbarrier wait of the tensor-core GEMM is bounded.  A wait that runs
 * out sets a device status word; the kernel then waits for its TMA loads in
 * flight and its tensor-core work, frees its tensor memory and returns without
 * writing its output tile.  chert_mlp_forward and chert_mlp_train_step read
 * the word after their work (synchronising the stream) and return
 * CHERT_ETIMEOUT if it was set, clearing it.
 *
 * chert_mlp_check reads and clears the word on its own (synchronises
 * `stream`): for callers that enqueue the surrogate under stream capture,
 * where nothing reads it.  Returns CHERT_OK or CHERT_ETIMEOUT.
 *
 * chert_mlp_set_wait_limit sets the poll limit of the GEMM's main-loop waits
 * (default 2^22; polls < 0 queries) and returns the previous one.  It exists
 * so that a test can make a wait run out (polls = 0) and check the status
 * and the fallback; process-wide, synchronous. */
int chert_mlp_check(void* stream);
long long chert_mlp_set_wait_limit(long long polls);

/* y [n][5] (standardised outputs) for x [n][8]; all device.  Errors:
 * CHERT_EINVAL, CHERT_ENOMEM (workspace), CHERT_ETIMEOUT (a tensor-core
 * wait ran out), CHERT_ECUDA. */
int chert_mlp_forward(const float* d_params, const float* d_x, int64_t n, float* d_y,
                      void* d_ws, size_t ws_bytes, void* stream);

/* One training step on a batch: loss = mean over samples of the halved
 * squared error of outputs 0, 1, 2, 4 against the standardised targets (valid
 * samples only) plus the logistic loss of output 3 against the validity in
 * t[:, 3]; t [n][5] holds raw targets, and a NaN target of output 0, 1, 2 or
 * 4 adds neither loss nor gradient.  Writes the gradient to d_grad_out
 * (may be NULL) and, if lr > 0, applies Adam (beta 0.9/0.999, eps 1e-8, bias
 * correction with step >= 1) to the trained part of d_params with moments
 * d_m, d_v.  d_loss (device float, may be NULL) receives the batch loss. */
int chert_mlp_train_step(float* d_params, float* d_m, float* d_v, int step, float lr,
                         const float* d_x, const float* d_t, int64_t n, float* d_loss,
                         float* d_grad_out, void* d_ws, size_t ws_bytes, void* stream);

/* Training pairs from an exact cache built by chert_build_cache with the same
 * classes and M: for every (class, folded angle j = 0..M) of cache mode slot
 * `mode_slot` (wave mode `mode`), features x [n][8] and raw targets t [n][5]
 * (n = n_classes*(M+1)); flagged entries get t[:, 3] = 0, and qSV entries
 * with |vartheta| > 2 deg NaN targets for outputs 0-2 (the surrogate hands
 * qSV entries beyond 1 deg to the exact solver, so only their validity and
 * vartheta are learnt).  d_scratch holds
 * at least 13*n bytes.  precision: storage type of the exact cache. */
int chert_surrogate_dataset(const chert_class* d_classes, int n_classes, int M, int mode,
                            int mode_slot, const chert_cache_arrays* exact, int precision,
                            float* d_x, float* d_t, void* d_scratch, size_t scratch_bytes,
                            void* stream);

/* A cache of the same layout and meaning as chert_build_cache's, filled by
 * the networks (d_params_per_mode: host array of n_modes device pointers).
 * flag = 0 valid, 1 no acceptable root (network), 2 needs the exact solver:
 * the medium lies outside the training range, the network is unsure whether
 * a decaying root exists (0.1 < p < 0.9), or, for qSV, the predicted
 * imaginary angle exceeds the fallback angle (chert_set_surrogate_qsv_angle,
 * 1 deg by default: the cusp / triplication region), and every solve if a
 * tensor-core GEMM wait ran out.  The caller recomputes those solves with
 * chert_build_cache_items, or calls chert_cache_surrogate, which does both.
 * Outside stream capture it reads the tensor-core status at the end (one
 * synchronisation; CHERT_ETIMEOUT if a wait ran out); under capture it does
 * not (chert_mlp_check). */
size_t chert_surrogate_cache_workspace_bytes(int n_classes, int M);

/* The qSV fallback angle of chert_surrogate_cache, process-wide: qSV entries
 * the network calls valid whose predicted imaginary angle exceeds `rad` get
 * flag 2 (exact solver); the default is 1 deg, 0 hands every such entry to
 * the exact solver.  rad < 0 queries.  Returns the previous (or current)
 * angle. */
double chert_set_surrogate_qsv_angle(double rad);
int chert_surrogate_cache(const float* const* d_params_per_mode, const chert_class* d_classes,
                          int n_classes, const int* modes, int n_modes, int M, int precision,
                          const chert_cache_arrays* out, void* d_ws, size_t ws_bytes,
                          void* stream);

/* The surrogate cache with its exact fallback in one enqueued sequence, no
 * host synchronisation (capturable into a CUDA graph): chert_surrogate_cache
 * (network precision CHERT_FP64 for an FP64 params->precision, else
 * CHERT_FP32), then the solves it marks with flag 2 are compacted on the
 * device into a list whose length stays on the device, and recomputed by the
 * exact solver (chert_build_cache_items' arithmetic at params: scan grid,
 * kernel, precision).  Every entry then has flag 0 or 1.  The tensor-core
 * status is not read here: if a GEMM wait ran out, every solve is marked for
 * and recomputed by the exact solver (a correct, slower cache), and
 * chert_mlp_check reports it.
 *   d_ws: device workspace of chert_cache_surrogate_workspace_bytes bytes.
 *   d_n_fallback: optional device int64, receives the number of solves
 *   recomputed exactly.
 * Errors: CHERT_EINVAL (counts, NULL), CHERT_ENOMEM (workspace), CHERT_ECUDA. */
size_t chert_cache_surrogate_workspace_bytes(int n_classes, int n_modes, int M);
int chert_cache_surrogate(const float* const* d_params_per_mode, const chert_class* d_classes,
                          int n_classes, const int* modes, int n_modes,
                          const chert_cache_params* params, const chert_cache_arrays* out,
                          void* d_ws, size_t ws_bytes, int64_t* d_n_fallback, void* stream);

/* The paper has no counterpart to this entry point; it exists for callers of
 * this library that cannot allocate device memory: code embedded in a host
 * whose device memory is all owned by the host's own pool, or a runtime that
 * forbids allocation after start-up.  It computes what chert_traveltime
 * computes, bit for bit, with the same arguments minus the workspace, and
 * allocates nothing: its scratch is a fixed 1 MiB array in device memory that
 * libchert declares at file scope, so every device that loads the library
 * holds that array until the process exits.
 *   - Problems whose scratch (chert_traveltime_workspace_bytes) exceeds
 *     chert_traveltime_static_limit() minus 256 bytes are rejected with
 *     CHERT_EINVAL and a message naming both sizes, before any output is
 *     touched.
 *   - On 2D lattices with too many classes for the class-pair table (e.g.
 *     one class per node), chert_traveltime with a lattice-sized workspace
 *     relaxes on precomputed per-node weights; here those weights use the
 *     rest of the array when they fit, and otherwise the generic kernel runs
 *     (same fields and parents, slower).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for the
 *     life of the process.  A cudaDeviceReset of that device invalidates it,
 *     so do not call this entry point on a device after resetting it.
 *   - It reads its status back and synchronises `stream`, so it cannot be
 *     called while that stream is being captured into a CUDA graph; use
 *     chert_traveltime_enqueue there.
 *   - All calls share the one array and it keeps the last call's contents
 *     (the parts that must start at zero are cleared by each call).  Calls
 *     that overlap on the GPU -- on different streams or from different host
 *     threads -- race on it: serialise them.
 * Errors: as chert_traveltime, CHERT_ENOMEM never. */
int chert_traveltime_static(const chert_cache_arrays* cache, int n_modes, int n_classes,
                            int n_dir, int nx, int ny, int nz, double dx,
                            const int32_t* d_class_of_node, const int32_t* offsets,
                            int n_off, const int64_t* sources, int n_sources,
                            int precision, int max_cycles,
                            void* d_tauR, void* d_tauI, int32_t* d_parR, int32_t* d_parI,
                            void* stream);

/* Size in bytes of chert_traveltime_static's scratch array. */
size_t chert_traveltime_static_limit(void);

/* ---- raypaths (Eq. 33-34) ------------------------------------------------ */

/* Backtrack parents from receivers to sources for a batch of fields.  Field
 * f has parents d_par[f*n_nodes ...] (int32, as written by chert_traveltime)
 * and source d_src[f]; for receiver r its path is written source-first to
 * d_paths[(f*n_rcv + r)*cap ...] and its node count to d_len[f*n_rcv + r],
 * 0 when the receiver is unreachable, a parent is out of range, or the walk
 * exceeds cap nodes (a cycle cannot run forever).  All arrays are device
 * memory: par int32 [n_fields][n_nodes], src int64 [n_fields], rcv int64
 * [n_rcv], paths int64 [n_fields][n_rcv][cap], len int64 [n_fields][n_rcv].
 * Errors: CHERT_EINVAL, CHERT_ECUDA. */
int chert_raypath(const int32_t* d_par, int n_fields, int64_t n_nodes,
                  const int64_t* d_src, const int64_t* d_rcv, int n_rcv, int64_t cap,
                  int64_t* d_paths, int64_t* d_len, void* stream);

/* Tie log of the parent rule (Eq. 33).  For converged fields (as returned by
 * chert_traveltime or chert_traveltime_enqueue for the same cache, lattice,
 * class map, stencil and sources), node j of field f and component c is a
 * tie when the second-best in-neighbour candidate tau_i + w_ij lies within
 * rel_tol * best of the best one: rounding at that level can then make either
 * predecessor the parent, so two correct implementations may return
 * different parents (and raypaths through j) there.  The source and
 * unreachable nodes are never ties.
 *   d_Vsel, d_Asel  device [n_modes][n_classes][n_off] lookup tables from
 *                   chert_edge_table (the relaxation's weights, Eq. 28-30, are
 *                   rebuilt from them with the same rounding); double for
 *                   CHERT_FP64, float otherwise
 *   d_tauR, d_tauI  device [n_sources][n_modes][nodes]: double for CHERT_FP64
 *                   and CHERT_FP32_ACC64, float otherwise
 *   d_tieR, d_tieI  device uint8 [n_sources][n_modes][nodes] (0/1), may be NULL
 *   d_counts        device uint64 [n_sources*n_modes][2] (ties per field and
 *                   component), may be NULL
 * Candidates are formed in the traveltime type; at most 65535 fields per
 * call.  Errors: CHERT_EINVAL, CHERT_ECUDA. */
int chert_parent_ties(const void* d_Vsel, const void* d_Asel, int n_modes, int n_classes, int precision,
                      int nx, int ny, int nz, double dx, const int32_t* d_class_of_node,
                      const int32_t* offsets, int n_off, const int64_t* d_sources, int n_sources,
                      const void* d_tauR, const void* d_tauI, double rel_tol, uint8_t* d_tieR,
                      uint8_t* d_tieI, unsigned long long* d_counts, void* stream);

/* ---- the whole path on host buffers (Algorithm 2) ------------------------- */

/* Device scratch bytes chert_trace_host needs (0 for invalid sizes). */
size_t chert_trace_host_scratch_bytes(int n_classes, int n_modes, int M, int nx, int nz, int n_off,
                                      int n_sources, int n_rcv, int64_t path_cap, int precision);

/* Algorithm 2 on a 2D lattice as one call on host buffers: copies the classes,
 * class map, sources and receivers to the device, builds the cache
 * (chert_build_cache with `params`; CHERT_FP64 gives double fields, CHERT_FP32
 * and CHERT_MIXED float ones), relaxes every (source, mode) field with parents
 * (chert_traveltime_enqueue), traces the raypaths of both components to every
 * receiver (chert_raypath), copies the traveltime fields and raypaths back,
 * and synchronises `stream` once.
 *   h_classes        host [n_classes]; modes host [n_modes]
 *   h_class_of_node  host int32 [nz*nx]; offsets host int32 [n_off][3] (oy = 0)
 *   h_sources        host int64 [n_sources]; h_receivers host int64 [n_rcv]
 *   h_tauR, h_tauI   host [n_sources][n_modes][nz*nx] (float or double)
 *   h_paths          host int64 [2][n_sources*n_modes][n_rcv][path_cap]
 *                    (component 0 = propagation, 1 = attenuation; source first)
 *   h_path_len       host int64 [2][n_sources*n_modes][n_rcv] (0: unreachable
 *                    or longer than path_cap)
 *   d_scratch        device, at least chert_trace_host_scratch_bytes()
 * The sources are relaxed in waves (the first fills two resident CTAs a SM
 * with its field components); each wave's fields and raypaths are copied
 * back on a copy stream while the next wave relaxes.  Host buffers should be
 * page-locked for the copies to run asynchronously at full speed.  Errors:
 * as the entry points it chains (a cycle cap names the first failing field
 * of the first wave that has one), CHERT_ENOMEM (scratch too small). */
int chert_trace_host(const chert_class* h_classes, int n_classes, const int* modes, int n_modes,
                     const chert_cache_params* params, int nx, int nz, double dx,
                     const int32_t* h_class_of_node, const int32_t* offsets, int n_off,
                     const int64_t* h_sources, int n_sources, int max_cycles, const int64_t* h_receivers,
                     int n_rcv, int64_t path_cap, void* h_tauR, void* h_tauI, int64_t* h_paths,
                     int64_t* h_path_len, void* d_scratch, size_t scratch_bytes, void* stream);

/* ---- measurement helpers (no counterpart in the paper) ---------------------- */

/* Measured multiply-add rate of this device in flop/s (2 per FMA), for the
 * roofline of the cache build: CTAs of 256 threads, 8 per SM, each thread
 * running 8 independent chains of `iters` FMAs in float (CHERT_FP32) or
 * double (CHERT_FP64), timed with events on `stream` (synchronises it).
 * Errors: CHERT_EINVAL, CHERT_ECUDA. */
int chert_fma_rate(int precision, int iters, double* flops_per_s, void* stream);

/* Counter of energy-velocity evaluations in the cache build (Eq. 12-14; one
 * per thread and evaluation: scan grid points, polish and refinement points,
 * ray quantities), process-wide, off by default.  enable = 1 zeroes the
 * counts and switches counting on for the current device; enable = 0
 * synchronises the device, switches it off and writes the counts of float,
 * float-float and double evaluations to counts_out[3] (may be NULL).
 * Counting adds one atomic per warp and evaluation; time builds with it off.
 * Errors: CHERT_ECUDA. */
int chert_cache_eval_counter(int enable, unsigned long long* counts_out);

/* Message describing the last error returned on the calling host thread. */
const char* chert_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CHERT_H */
