/*
 * pd.h -- C ABI of the localized-collision Projective Dynamics library
 * (Wang, Tao, Brandt, Cutting, Sifakis, "Optimized Processing of Localized
 * Collisions in Projective Dynamics", SCA 2020).
 *
 * One solver handle owns one scene on one CUDA device.  Every entry point
 * returns a pd_status; the library never aborts or exits.  On any error the
 * handle stays usable, the solver state is left as it was before the call,
 * and pd_last_error() describes what happened.
 *
 * Conventions
 *   - Host pointers are read (or written) during the call only; the caller
 *     keeps ownership.  Entry points ending in _dev take device pointers that
 *     must stay valid until the call returns on the solver's stream.
 *   - Node ids and element indices are int32 and 0-based; sizes are int64.
 *   - Positions are [n][3] row-major float64 in the caller's node order.
 *   - The solver owns all device memory it allocates and frees it in
 *     pd_destroy().
 */
#ifndef PD_H
#define PD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PD_OK = 0,
    PD_ERR_INVALID_ARG = 1,            /* null pointer, negative size, bad option   */
    PD_ERR_BAD_MESH = 2,               /* degenerate rest tet or node id out of range */
    PD_ERR_REGION = 3,                 /* region empty, overlaps Dirichlet, or too large */
    PD_ERR_CONTACT_OUTSIDE_REGION = 4, /* a contact names a node outside x_2        */
    PD_ERR_NOT_SPD = 5,                /* a Cholesky pivot was not positive         */
    PD_ERR_NO_CONVERGENCE = 6,         /* refinement / PCG missed tol in max_refine */
    PD_ERR_TIMEOUT = 7,                /* a bounded device wait gave up             */
    PD_ERR_CUDA = 8,                   /* a CUDA runtime call failed                */
    PD_ERR_OOM = 9                     /* device or host allocation failed          */
} pd_status;

/* Precision of the collision-region solve H u_2 = g (Algorithm 1, step 4.5). */
enum {
    PD_FP64 = 0,      /* FP64 blocked Cholesky of H and FP64 triangular solves      */
    PD_FP32_IR = 1,   /* FP32 factor (split-TF32 tensor-core updates), iterative
                         refinement with FP64-accurate residuals                    */
    PD_TF32_IR = 2,   /* TF32 tensor-core trailing updates, CG refinement with
                         FP64-accurate residuals                                   */
    PD_BF16_IR = 3,   /* BF16 tensor-core trailing updates, CG refinement with
                         FP64-accurate residuals                                   */
    /* FP64-accurate residual r = g - H u: FP64 vectors, Sigma_0 u from Sigma_0
     * held as an FP32 head + tail pair (~48 bits) in double-float arithmetic,
     * the contact term C_22 u in FP64.                                         */
    PD_PCG_WARM = 4   /* PCG on H preconditioned by the contact-free factor of Sigma,
                         started from a caller-supplied (e.g. learned) guess; the
                         preconditioner carries the active springs exactly through
                         a capacitance (Woodbury) correction unless
                         pd_set_pcg_capacitance turns it off                        */
};

typedef struct {
    int64_t n_nodes;
    const double* rest_pos;   /* [n_nodes][3] */
    int64_t n_tets;
    const int32_t* tets;      /* [n_tets][4], either orientation */
} pd_mesh;

typedef struct {
    double mu;        /* Lame mu of the PD energy mu ||F - R||_F^2 (Eq. 2)       */
    double lambda;    /* accepted and ignored: the method sets lambda = 0 (Sec 2.2);
                         its PD counterpart is the volume term kappa below     */
    double density;   /* used for the lumped mass when dt > 0                    */
    /* Bi-phasic strain limiting (Section 5): the energy density gains
     * mu_prime * min_{Q in S} ||F - Q||_F^2, S = the matrices whose singular
     * values lie in [sigma_min, sigma_max] (the paper's open set, taken with
     * its closure).  mu_prime = 0 (zero-initialised struct) turns it off;
     * otherwise 0 <= sigma_min <= sigma_max (sigma_max may be +inf).  The
     * system matrix then carries mu + mu_prime for every element.           */
    double mu_prime;
    double sigma_min, sigma_max;
    /* PD volume term (the lambda term of Eq. 1, (lambda/2) tr^2(S - I), has
     * no PD form: with R fixed its Hessian depends on R): the energy density
     * gains kappa * ||F - T||_F^2, T the matrix nearest F with
     * det T in [det_min, det_max], found from the signed SVD of F on the
     * principal branch of the stationarity condition (the nearest such
     * matrix for every contraction and inversion, and for expansions up to
     * about 1.9x in every direction).  With det_min = det_max = 1 and
     * kappa = 3 lambda / 2 it agrees with the lambda term to second order
     * in the strain.  kappa = 0 (zero-initialised struct) turns it off;
     * otherwise 0 < det_min <= det_max (det_max may be +inf).  The system
     * matrix then carries mu + mu_prime + kappa for every element.        */
    double kappa;
    double det_min, det_max;
} pd_material;

typedef struct {
    int precision;     /* PD_FP64, PD_FP32_IR, ... (default PD_FP64)            */
    double tol;        /* relative residual ||g - H u|| / ||g|| for the refined forms (1e-10) */
    int max_refine;    /* refinement / PCG iteration cap (default 50)           */
    int inner_iters;   /* inner iterations per outer iteration (Algorithm 1, step 4) */
    void* cuda_stream; /* cudaStream_t to run on; NULL = the library's own stream */
    int timing;        /* nonzero: record CUDA events per phase (pd_get_stats)  */
} pd_options;

typedef struct {
    int64_t n_nodes, n_tets, n_free, n1, m;   /* sizes after partitioning            */
    int64_t n_alpha, n_beta;                  /* |E_alpha|, |E_beta|                 */
    int64_t n_supernodes, n_levels, nnz_L;    /* interior factor L_1 and L_21        */
    int64_t contacts;                         /* active springs in the last inner iteration */
    int64_t outer_done, inner_done;           /* iterations run by the last pd_step  */
    int refine_iters;                         /* refinement / PCG iterations: summed over the
                                                 solves of the last pd_step, or of the last
                                                 pd_schur_solve */
    double residual;                          /* ||g - H u|| / ||g|| of the last solve
                                                 (-1: not measured, the direct FP64 form) */
    double setup_ms;                          /* wall time of pd_setup               */
    /* per-phase device time of the last pd_step (timing != 0), milliseconds:      */
    double ms_local_alpha;    /* a1: alpha polar + forces + gather                  */
    double ms_forward;        /* a2: sparse forward substitution                    */
    double ms_contact_update; /* a3: H = Sigma_0 + C_22                             */
    double ms_local_beta;     /* a4: beta polar + forces + RHS g                    */
    double ms_factor_solve;   /* a5: refactor + solve (incl. refinement)            */
    double ms_bookkeeping;    /* a6: x_2 += u_2, f~_2 -= Sigma_alpha u_2             */
    double ms_backward;       /* a7: sparse backward substitution                   */
    double ms_step;           /* whole pd_step                                      */
    int64_t kernel_launches;  /* kernels this library launched during the last pd_step */
    double ms_refactor;       /* the refactorisation alone (part of ms_factor_solve; PCG forms: 0) */
    int64_t starts_rejected;  /* supplied PCG starts replaced by zero since pd_setup
                                 (see pd_set_warm_start)                              */
    int64_t precision_fallbacks; /* low-precision solves redone in FP64 since pd_setup
                                    (see pd_set_precision_fallback)                   */
} pd_stats;

typedef struct pd_solver pd_solver;

/* Called once per inner iteration (Algorithm 1, step 4.1, DetectCollisions)
 * with the current collision-prone positions x2 [m][3] (host, region order).
 * It may call pd_set_contacts() on the solver; a non-PD_OK return aborts the
 * step (state rolled back) and is returned by pd_step. */
typedef pd_status (*pd_contact_cb)(void* user, const double* x2, pd_solver* s);

/* Build a solver (Algorithm 1, "preliminary"): element rest data, the node
 * split into x_1 / x_2 and E_alpha / E_beta (Section 3.4, Figure 2), the
 * interior ordering (nested dissection, x_2 last: Section 3.2), the partial
 * Cholesky A = [L_1 0; A_21 L_1^-T I] diag(I, Sigma_alpha) [...]^T of the
 * alpha matrix (Eq. 9) and Sigma_0 = Sigma_alpha + A_22^beta (+ M_2/dt^2).
 *   mesh, mat     : rest mesh and material (copied)
 *   dt            : time step; 0 = quasistatic (Eq. 4), > 0 = backward Euler
 *   region, m     : the m collision-prone node ids x_2 (any order; row i of
 *                   Sigma is region[i]); 1 <= m <= 16384
 *   dirichlet, nd : fixed node ids; must not meet the region
 *   opts          : may be NULL for defaults
 *   out           : receives the handle; NULL on failure
 * Errors: INVALID_ARG, BAD_MESH, REGION, NOT_SPD (a free component without a
 * Dirichlet node in quasistatic mode), CUDA, OOM. */
pd_status pd_setup(const pd_mesh* mesh, const pd_material* mat, double dt,
                   const int32_t* region, int64_t m,
                   const int32_t* dirichlet, int64_t nd,
                   const pd_options* opts, pd_solver** out);

/* Prescribe the Dirichlet positions [nd][3] (order of pd_setup's list);
 * they take effect at the next pd_step.  Errors: INVALID_ARG. */
pd_status pd_set_dirichlet(pd_solver* s, const double* pos);

/* Replace the active penalty springs (Section 2.3, Eqs. 6-8): spring j pulls
 * the proxy p_j = sum_a w[j][a] x[nodes[j][a]] toward target[j] with stiffness
 * stiffness[j]; unused slots have nodes = -1 and w = 0.  Every named node must
 * lie in x_2.  k = 0 clears all springs.  Errors: INVALID_ARG,
 * CONTACT_OUTSIDE_REGION (state unchanged), CUDA, OOM. */
pd_status pd_set_contacts(pd_solver* s, int64_t k, const int32_t* nodes /*[k][4]*/,
                          const double* w /*[k][4]*/, const double* target /*[k][3]*/,
                          const double* stiffness /*[k]*/);

/* Two-sided springs between two proxies (self-collision, Section 2.3 with
 * the spring between p_a and p_b; the paper notes that W is re-sent for
 * self-collision, Section 3.3): spring j acts on the difference
 * d_j = sum_{a<8} w[j][a] x[nodes[j][a]] -- typically slots 0..3 hold one
 * proxy's barycentric weights and slots 4..7 the other's, negated -- with
 * energy stiffness[j]/2 ||d_j - target[j]||^2 (target = the separation to
 * keep, frozen for the iteration).  Same ownership and errors as
 * pd_set_contacts; replaces all springs. */
pd_status pd_set_contact_pairs(pd_solver* s, int64_t k, const int32_t* nodes /*[k][8]*/,
                               const double* w /*[k][8]*/, const double* target /*[k][3]*/,
                               const double* stiffness /*[k]*/);

/* Collision detection on the device (Algorithm 1, step 4.1, run at every
 * inner iteration when pd_step gets no callback).  Each proxy (or side-A
 * proxy) owns one spring slot; inactive proxies contribute nothing.
 * Spheres: proxies [np] (node ids in x_2) inside a rigid sphere spheres[q] =
 * {cx, cy, cz, r} get a zero-rest-length spring of stiffness `stiffness` to
 * their projection on the deepest sphere's surface.
 * Pairs: each side-A node within `gap` of its nearest side-B node gets a
 * two-sided spring on x_a - x_b toward separation `gap` (self-collision).
 * While a detector is set, pd_step without a callback re-detects at every
 * inner iteration and so replaces springs given by pd_set_contacts; with a
 * callback the callback's springs are used.  pd_clear_detector removes the
 * detector and all springs.  The detector's arrays are copied; the caller
 * keeps ownership of its buffers.
 * Errors: INVALID_ARG (negative counts, null arrays, non-finite values,
 * gap <= 0), CONTACT_OUTSIDE_REGION (a node not in x_2), CUDA. */
pd_status pd_set_detector_spheres(pd_solver* s, const int32_t* proxies, int64_t np, int nsph,
                                  const double* spheres /*[nsph][4]*/, double stiffness);
pd_status pd_set_detector_pairs(pd_solver* s, const int32_t* side_a, int64_t na, const int32_t* side_b,
                                int64_t nb, double gap, double stiffness);
/* Point-triangle self-contact on the device (Algorithm 1, step 4.1; the
 * paper's proxies are barycentric points of surface elements, Section 3.1):
 * each side-A proxy node is tested against the side-B surface triangles
 * tris_b [ntb][3] (node ids, wound so that (b - a) x (c - a) is the outward
 * normal), and each side-B proxy against tris_a [nta][3].  A node skips the
 * triangles that lay within rest_min of it in the rest pose (the surface
 * around it, e.g. across the crease where the two sides meet), takes the
 * nearest remaining triangle (lowest index on ties) and, if its closest
 * point q is nearer than gap, gets a two-sided spring on x_node - q (q = the
 * barycentric combination of the triangle's nodes: slots 0 and 4..6 of the
 * 8-slot row) of the given stiffness toward gap * n, n the triangle's unit
 * normal at detection, i.e. the node is pushed to the surface offset by gap
 * in front of q.  One spring slot per proxy (na + nb); inactive proxies
 * contribute nothing.  Every node named must lie in x_2.  The arrays are
 * copied.  Errors: INVALID_ARG (negative counts, null arrays, gap <= 0,
 * rest_min < 0, non-finite values), CONTACT_OUTSIDE_REGION, CUDA. */
pd_status pd_set_detector_triangles(pd_solver* s, const int32_t* prox_a, int64_t na, const int32_t* tris_a,
                                    int64_t nta, const int32_t* prox_b, int64_t nb, const int32_t* tris_b,
                                    int64_t ntb, double gap, double rest_min, double stiffness);
pd_status pd_clear_detector(pd_solver* s);

/* Run the device detector once on the current positions (Algorithm 1, step
 * 4.1 alone, no solve); its springs become the active ones, as they would at
 * the start of an inner iteration.  Synchronous.  Errors: INVALID_ARG (no
 * detector set), CUDA. */
pd_status pd_detect(pd_solver* s);

/* Read back the active spring slots (as pd_set_contact_pairs takes them:
 * [k][8] node ids with -1 in unused slots, weights, targets [k][3],
 * stiffness [k]; a detector's inactive slots have stiffness 0 and no nodes).
 * *k receives the number of slots; at most cap are copied.  Synchronous.
 * Errors: INVALID_ARG, CUDA. */
pd_status pd_get_contacts(const pd_solver* s, int64_t cap, int64_t* k, int32_t* nodes /*[cap][8]*/,
                          double* w /*[cap][8]*/, double* target /*[cap][3]*/, double* stiffness /*[cap]*/);

/* Declare the region nodes that springs may touch (FP64 form).  H = Sigma_0
 * + C_22 has C_22 = 0 outside those rows and columns, so the region is
 * ordered with the other nodes first, the partial Cholesky of those leading
 * rows (in whole 64-row tiles) is computed once here, and every
 * refactorisation (Algorithm 1, 4.3-4.5) factors only the trailing block
 * S_p + C_pp, S_p being the Schur complement of the fixed rows; the solve is
 * the same H u = g in FP64.  Springs set earlier and the device detector are
 * dropped; later springs (pd_set_contacts, detectors) may touch only these
 * nodes.  np = 0 turns it off.  The nested Schur complement is this
 * library's; the paper refactors all of H.
 * Errors: INVALID_ARG, CONTACT_OUTSIDE_REGION (a node not in x_2), NOT_SPD,
 * CUDA, OOM. */
pd_status pd_set_contact_nodes(pd_solver* s, const int32_t* nodes, int64_t np);

/* One time step: outer_iters passes of Algorithm 1 (Section 3.4).  If cb is
 * not NULL it is called at every inner iteration before the local beta step;
 * otherwise the springs last set stay active.  Errors: NOT_SPD,
 * NO_CONVERGENCE, TIMEOUT, CUDA, or the callback's status; on error the
 * positions and velocities are those from before the call. */
pd_status pd_step(pd_solver* s, int outer_iters, pd_contact_cb cb, void* user);

/* Current positions [n][3] (host). */
pd_status pd_get_positions(const pd_solver* s, double* out);

/* Current positions into a caller-owned device buffer [n][3]. */
pd_status pd_get_positions_dev(const pd_solver* s, double* out_dev);

/* Checkpoint / restore: positions and velocities [n][3] (host); v may be NULL
 * (quasistatic). */
pd_status pd_get_state(const pd_solver* s, double* x, double* v);
pd_status pd_set_state(pd_solver* s, const double* x, const double* v);

/* Counters and per-phase timings of the last pd_step. */
pd_status pd_get_stats(const pd_solver* s, pd_stats* out);

/* Text of the last error on this handle ("" if none).  Valid until the next
 * call on the handle.  s may be NULL for errors of pd_setup. */
const char* pd_last_error(const pd_solver* s);

/* Free the handle and every device buffer it owns.  NULL is ignored. */
void pd_destroy(pd_solver* s);

/* ------------------------------------------------------------------------
 * Kernel-level entry points (used by the parity tests and the benchmark).
 * ------------------------------------------------------------------------ */

/* Local step on all elements (Section 2.2): for each tet e, R_e = polar(F_e)
 * in SO(3) with F_e = Ds Dm^-1 at positions x [n][3] (host), and the elastic
 * forces f = -dE_hat/dx, f_e = -Vol_e 2 mu (F_e - R_e) G_e^T, summed per node;
 * with strain limiting f_e gains -Vol_e 2 mu' (F_e - Q_e) G_e^T (Section 5).
 *   R_out : [n_tets][3][3] row-major (host), may be NULL
 *   f_out : [n][3] (host), may be NULL; Dirichlet nodes receive their sums too */
pd_status pd_local_step(pd_solver* s, const double* x, double* R_out, double* f_out);

/* Sigma_0 = Sigma_alpha + A_22^beta (+ M_2/dt^2), dense [m][m] row-major,
 * region order (host). */
pd_status pd_get_schur(const pd_solver* s, double* out);

/* Schur refactor + solve (Algorithm 1, steps 4.3 and 4.5, Section 3.3): form
 * H = Sigma_0 + C_22 from the springs last set with pd_set_contacts, factor
 * it in the solver's precision and solve H u = g for three right-hand sides.
 *   g : [m][3] host (region order);  u : [m][3] host output
 *   u0: [m][3] host initial guess for PD_PCG_WARM, may be NULL (zero)
 * Errors: NOT_SPD, NO_CONVERGENCE, CUDA. */
pd_status pd_schur_solve(pd_solver* s, const double* g, const double* u0, double* u);

/* Same on device buffers (g_dev, u_dev [m][3]; u0_dev may be NULL). */
pd_status pd_schur_solve_dev(pd_solver* s, const double* g_dev, const double* u0_dev, double* u_dev);

/* Host-only partial Cholesky (no device needed): runs the setup of pd_setup
 * on the CPU and returns Sigma_0 (dense [m][m] row-major, region order) and
 * a one-line summary of the factorisation in info (may be NULL; at most
 * info_len bytes including the terminating zero).  Same arguments and errors
 * as pd_setup (Algorithm 1 "preliminary", Eq. 9). */
pd_status pd_host_schur(const pd_mesh* mesh, const pd_material* mat, double dt,
                        const int32_t* region, int64_t m,
                        const int32_t* dirichlet, int64_t nd,
                        double* sigma_out, char* info, int64_t info_len);

/* Allocation-free Schur refactor + solve (FP64).  The paper has no
 * counterpart: this exists for callers that may not allocate device memory
 * while they run -- an engine that reserves all of the GPU's memory up front
 * and forbids cudaMalloc/cudaFree mid-frame, an arena/pool integration, or a
 * real-time loop that cannot take the synchronisation an allocation implies.
 * It computes the same result as pd_schur_solve_dev() in PD_FP64 mode, but
 * without a solver handle and without allocating: its working memory is one
 * file-scope device array of about 8.5 MB that every device which loads this
 * library holds until the process exits.
 *   sigma_dev : [m][m] device, the symmetric Sigma_0 (row- or column-major)
 *   m         : 1 <= m <= 1024; larger m returns PD_ERR_INVALID_ARG
 *   k, cidx_dev [k][4], cw_dev [k][4], cs_dev [k] : springs on region rows
 *               (cidx = -1 marks an unused slot); H = Sigma_0 + sum_j c_j w_j w_j^T
 *   g_dev, u_dev : [m][3] device right-hand sides and solution
 *   cuda_stream  : stream to run on (NULL = the default stream)
 *   err, err_len : optional buffer for a message
 * The call is synchronous: it copies the contact indices and the pivot
 * status back to the host and waits for its stream, so it must not be issued
 * while that stream is being captured.  The first call on each device also
 * looks up the scratch array's device address.  All calls share the one
 * array, which keeps the last call's contents (the call rewrites everything
 * it reads), so calls that overlap on the GPU (other threads, other streams)
 * race.
 * Errors: INVALID_ARG, CONTACT_OUTSIDE_REGION, NOT_SPD, CUDA. */
pd_status pd_schur_solve_noalloc(const double* sigma_dev, int64_t m, int64_t k,
                                 const int32_t* cidx_dev, const double* cw_dev, const double* cs_dev,
                                 const double* g_dev, double* u_dev, void* cuda_stream,
                                 char* err, int64_t err_len);

/* Tensor-core rank-K update, exposed for diagnostics: C -= A B^T with A [M][K],
 * B [N][K], C [M][N] row-major float32 device buffers, M and N multiples of 128,
 * K = 128.  mode 0 = TF32, 1 = split TF32 (three products, ~FP32 accuracy),
 * 2 = BF16 (operands rounded to bfloat16); accumulation is FP32 in tensor
 * memory.  This is the trailing-update kernel of the low-precision Cholesky
 * (Section 3.3 dense refactorisation).  Errors: INVALID_ARG, OOM, CUDA, TIMEOUT. */
pd_status pd_tc_rank_k(int mode, const float* A, const float* B, float* C, int64_t M, int64_t N, int64_t K,
                       void* cuda_stream);

/* ------------------------------------------------------------------------
 * Learned warm start for PD_PCG_WARM (beyond the paper: a small network that
 * predicts the collision-region solution u_2 of H u_2 = g, used only as the
 * starting point of PCG; the refined answer still has to meet tol).
 * The start is u0 = z0 + s * N(features), where z0 = M0^-1 g is the
 * response of the contact-free factor M0 of Sigma_0 (one preconditioner
 * application) and the network N predicts the contact correction u - z0.
 * Per region node, 14 inputs -- g_i / rms(g), z0_i / s, |g_i| / rms(g),
 * |z0_i| / s, contact flag, log(1 + contact stiffness / mean diag Sigma_0),
 * spring direction (3), normalised rest height -- then 256-256-256 ReLU
 * layers and 3 outputs; s = rms(g) / mean(diag Sigma_0).  BF16 weights and
 * activations, FP32 accumulation, all products on the tensor cores.
 * Parameter vector (float32, logical layout, 136195 values):
 *   W1 [256][14] b1 [256] W2 [256][256] b2 [256] W3 [256][256] b3 [256] W4 [3][256] b4 [3]
 * ------------------------------------------------------------------------ */
#define PD_MLP_NPARAMS 136195

/* Starting point of PD_PCG_WARM solves inside pd_step: 0 = zero, 1 = the
 * previous region solution, 2 = the network's prediction z0 + s N (needs
 * parameters), 3 = z0 alone (the contact-free response, no network).  A
 * start u0 (here or through pd_schur_solve's u0) is kept only when it lowers
 * the energy PCG minimises, phi(u) = u^T H u / 2 - g^T u, below phi(0) = 0,
 * i.e. when it is closer to the solution than zero in the H-norm; any other
 * start (or a non-finite one) is replaced by zero and counted in
 * pd_stats.starts_rejected, so a poor prediction never starts PCG farther
 * from the answer than the cold start. */
pd_status pd_set_warm_start(pd_solver* s, int source);

/* Capacitance correction of the PD_PCG_WARM preconditioner (beyond the
 * paper; on by default).  M0 (the FP32 factor of the contact-free Sigma_0,
 * Section 3.3) leaves one outlier eigenvalue of M0^-1 H per active spring.
 * With the correction, each refactorisation step instead gathers the k
 * active springs' rows V = C^1/2 W, forms Y = V M0^-1 and the k x k matrix
 * S = I + V M0^-1 V^T, and factors S in FP64; each PCG iteration then
 * applies P^-1 r = M0^-1 r - Y^T S^-1 V M0^-1 r (the Woodbury identity for
 * P = M0 + W^T C W).  The solve still meets tol against the FP64-accurate
 * residual of H.  on = 0 uses M0 alone.  Errors: INVALID_ARG (NULL s). */
pd_status pd_set_pcg_capacitance(pd_solver* s, int on);

/* Precision escalation of the low-precision forms (beyond the paper; on by
 * default).  A region solve of PD_FP32_IR, PD_TF32_IR, PD_BF16_IR or
 * PD_PCG_WARM whose low-precision factor lost a pivot (the pivot was not
 * positive and the refinement did not reach tol), or whose refinement did not
 * reach tol within max_refine, is redone for that system by the FP64
 * factorisation and direct solve of the same H (Section 3.3), and counted in
 * pd_stats.precision_fallbacks; the next refactorisation is low precision
 * again.  Not applied with pd_set_contact_nodes (the nested form), nor when H
 * itself has a non-positive diagonal entry.  If the FP64 factorisation fails
 * too, the step reports PD_ERR_NOT_SPD as the FP64 form does.  on = 0 reports
 * the low-precision failure (PD_ERR_NOT_SPD or PD_ERR_NO_CONVERGENCE) at once.
 * Errors: INVALID_ARG (NULL s). */
pd_status pd_set_precision_fallback(pd_solver* s, int on);

/* Set / read the network parameters (n must be PD_MLP_NPARAMS); setting them
 * resets the optimiser state. */
pd_status pd_mlp_set_params(pd_solver* s, const float* params, int64_t n);
pd_status pd_mlp_get_params(pd_solver* s, float* params, int64_t n);

/* Record (features, solution) pairs of the next max_solves region solves run
 * by pd_step / pd_schur_solve, on the device (the training set is generated
 * by the method itself).  0 stops recording.  Recording restarts the set. */
pd_status pd_mlp_record(pd_solver* s, int64_t max_solves);

/* Training loss: 0 = mean squared error of the correction (the default);
 * 1 = every node row weighted by H_ii / mean diag(Sigma_0), H_ii = Sigma_0[i][i]
 * + C_22[i][i] of the recorded solve: the diagonal of the energy norm
 * (u - u*)^T H (u - u*) that CG minimises, exact for the contact term of
 * single-node springs, so errors at the stiff spring nodes count as much as
 * they cost PCG.  pd_mlp_eval reports the same weighting.  Errors: INVALID_ARG. */
pd_status pd_mlp_set_loss(pd_solver* s, int kind);

/* Adam (lr, beta 0.9/0.999) on the training loss over `steps` minibatches
 * of `batch` recorded node rows (multiple of 128, <= 8192) drawn with a
 * counter-based generator from `seed`.  *loss = mean loss of the last steps. */
pd_status pd_mlp_train(pd_solver* s, int64_t steps, int64_t batch, double lr, uint64_t seed, double* loss);

/* Mean squared error on every recorded row of the network's correction,
 * against the true u - z0, and that of the zero correction (the z0 start),
 * in the scaled units: 1 - mse_net / mse_zero is the part of the remaining
 * error after the contact-free response that the network predicts. */
pd_status pd_mlp_eval(pd_solver* s, double* mse_net, double* mse_zero);

/* Loss and gradient (logical layout) at the current parameters for a host
 * batch X [B][14], T [B][3] (for checking the hand-written backward pass). */
pd_status pd_mlp_loss_grad(pd_solver* s, const float* X, const float* T, int64_t B, double* loss, float* grad);

/* Failure-detection check (no counterpart in the paper): launches a kernel
 * whose bounded wait on a flag that nothing sets gives up after a short poll
 * limit (~20 ms), and reports it the way every bounded device wait in the
 * library does.  Returns PD_ERR_TIMEOUT with the handle still usable. */
pd_status pd_debug_wait_timeout(pd_solver* s);

/* Change the precision of the collision-region solve on an existing handle. */
pd_status pd_set_precision(pd_solver* s, int precision);
/* Inner iterations per outer iteration (Algorithm 1, step 4), from the next
 * pd_step on.  Errors: INVALID_ARG (inner_iters < 1). */
pd_status pd_set_inner_iters(pd_solver* s, int inner_iters);

#ifdef __cplusplus
}
#endif
#endif /* PD_H */
