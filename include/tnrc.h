/*
 * tnrc -- tensor-network robust control on one GPU (C ABI).
 *
 * Computes, for the qubit chain of Eq. sysH with parasitic nearest-neighbour
 * ZZ crosstalk, the ensemble-averaged state fidelity
 *
 *     F = 1/(M P) sum_{s,p} | <t_p | U^(s) | in_p> |^2          (Sec. II; F = 1 - infidelity)
 *
 * over M noise realisations s (Sec. II: J_b^(s) iid per bond) and P input /
 * target state pairs, with U^(s) the TEBD evolution of K piecewise-constant
 * control slices (Sec. II, Eq. circuit; second or first order) on a complex128
 * matrix-product state truncated by SVD to bond dimension chi_max, and its
 * exact costate gradient dF/du with respect to every control amplitude
 * (App. A).
 *
 * Conventions shared by every entry point
 *   - Sites i = 0..N-1, bonds b = 0..N-2 (bond b couples sites b, b+1).
 *     |0> = (1,0) is the Z = +1 state.
 *   - Controls u[K][C][N] (float64, row-major): slot 0 = x_i, slot 1 = y_i
 *     (X / Y drives of site i), slot 2 (C = 3) = g_i, the tunable ZZ coupling
 *     of bond (i, i+1).  A slot whose control_mask entry is 0 is not a
 *     control: it does not enter the Hamiltonian and its gradient is 0.
 *   - Slice (control bin) k of length dt holds n_sub = substeps Trotter steps
 *     of length dts = dt / n_sub.  Second order (trotter_order 2, default):
 *     each step applies A(dts/2) B(dts) A(dts/2): A = the gates exp(-i tau h_b)
 *     of all even bonds, B = of all odd bonds, with
 *       h_b = (g_b + gfix_b + J^z_b) ZZ + J^x_b XX + J^y_b YY
 *             + wL (x_b X + y_b Y) (x) I + wR I (x) (x_{b+1} X + y_{b+1} Y),
 *     (J^x = J^y = 0 unless crosstalk_terms = 3),
 *     wL = 1 on bond 0 else 1/2, wR = 1 on bond N-2 else 1/2; the half steps
 *     A that meet at a step boundary are applied as one gate.  First order
 *     (trotter_order 1, the slice of Eq. circuit): each step applies
 *     exp(-i dts V_b) on every bond (odd bonds, then even bonds;
 *     V_b = (g_b + gfix_b + J^z_b) ZZ + J^x_b XX + J^y_b YY), then
 *     exp(-i dts y_i Y) and then exp(-i dts x_i X) on every site; each site's
 *     rotations are applied together with the last bond gate of the step that
 *     touches the site.
 *   - Truncation: after every two-site gate keep the
 *     k = min(chi_max, #{sigma_i > max(sv_cutoff, 1e-13) sigma_1}) largest
 *     singular values (at least one) and renormalise them to unit norm.
 *   - MPS buffers (tnrc_mps.data): interleaved complex128, site-major, site i
 *     stored as a row-major [D_i][d][D_{i+1}] block (d = 2, or 4 with
 *     operator_form); bond_dims has N+1 entries with bond_dims[0] =
 *     bond_dims[N] = 1.  States are normalised on entry.
 *   - Ownership: every host pointer passed in is borrowed for the duration of
 *     the call and copied; the context owns all device memory it uses.
 *     Output host buffers are written only when the call returns TNRC_OK.
 *   - Calls without the _dev suffix are ordered on the context's stream and
 *     synchronous at return.  One host thread per context at a time.
 *   - Errors: nothing aborts, traps or exits.  TNRC_E_CUDA leaves the context
 *     unusable (destroy it); every other error leaves it usable.
 */
#ifndef TNRC_H
#define TNRC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tnrc_status;
#define TNRC_OK 0
#define TNRC_E_INVALID (-1)   /* bad argument: NULL, size mismatch, out-of-range value  */
#define TNRC_E_NOMEM (-2)     /* device memory for the context could not be reserved    */
#define TNRC_E_CUDA (-3)      /* a CUDA call failed; the context is unusable             */
#define TNRC_E_STATE (-4)     /* controls or noise not set yet                           */
#define TNRC_E_TIMEOUT (-5)   /* a bounded device wait gave up (pooled launch)           */
#define TNRC_E_NUMERIC (-6)   /* Jacobi SVD did not converge, or a NaN/Inf appeared      */
#define TNRC_E_TOO_LARGE (-7) /* problem exceeds the fixed scratch of tnrc_fidelity_static */

typedef struct tnrc_ctx tnrc_ctx;

/* A matrix-product state (layout above).  n_sites must equal the problem's N. */
typedef struct {
  int32_t n_sites;
  const int32_t* bond_dims; /* [N+1] */
  const double* data;       /* interleaved complex128, sum_i D_i*d*D_{i+1} values */
} tnrc_mps;

/* The problem statement (Sec. II-IV): chain, time grid, truncation, ensemble. */
typedef struct {
  uint32_t struct_size;          /* sizeof(tnrc_problem)                                   */
  int32_t n_sites;               /* N >= 2                                                 */
  int32_t n_slices;              /* K >= 1 piecewise-constant control bins                 */
  double dt;                     /* slice length (> 0)                                     */
  int32_t chi_max;               /* bond-dimension cap, 1 <= chi_max <= 64 (<= 32 with
                                    operator_form)                                          */
  double sv_cutoff;              /* relative singular-value cutoff (>= 0; 1e-12 typical)   */
  int32_t n_samples;             /* M >= 1 noise realisations                              */
  int32_t n_controls;            /* C = 2 (x, y) or 3 (x, y, g)                             */
  int32_t n_inputs;              /* P >= 1 input/target pairs                              */
  const uint8_t* control_mask;   /* [C][N], 1 = control; NULL = all x, y (and g on bonds)  */
  const double* g_fixed;         /* [K][N-1] fixed ZZ added on every bond, or NULL         */
  int32_t checkpoint_every;      /* slices per backward segment when the forward history is
                                    recomputed; 0 = about sqrt(layers) truncated layers      */
  int32_t warps_per_cta;         /* trajectory-kernel warps per CTA, 2..8; 0 = default      */
  int32_t ctas_per_sm;           /* resident trajectory CTAs per SM, 1..4, clamped to
                                    warps_per_cta * ctas_per_sm <= 16; above 8 warps per SM
                                    the kernel's 128-register build runs; 0 = 1             */
  int32_t crosstalk_terms;       /* 1 (or 0): J^z ZZ per bond, J[M][N-1]; 3: the Heisenberg
                                    type J^x XX + J^y YY + J^z ZZ of Eq. Hp, J[M][N-1][3]
                                    in the order (x, y, z)                                 */
  int32_t trotter_order;         /* 2 (or 0): A(dts/2) B(dts) A(dts/2); 1: Eq. circuit      */
  int32_t substeps;              /* Trotter steps per slice, >= 1 (0 = 1)                   */
  int32_t operator_form;         /* 0: inputs/targets are states (physical dimension 2);
                                    1: they are operators written as vectors (MPO of Sec. II,
                                    physical dimension 4, site index s = 2 out + in, scaled so
                                    that <<A|B>> = tr(A^dag B) / 2^N); every gate acts as
                                    G (x) I on the out indices, so with input = the identity
                                    O = tr(U_T^dag U) / 2^N and F is one minus the gate
                                    infidelity of Eq. gateinfid                             */
} tnrc_problem;

/* Per-call statistics of the last tnrc_fidelity / tnrc_fidelity_grad. */
typedef struct {
  int64_t updates;               /* two-site updates executed (forward, recompute, costate) */
  int64_t jacobi_sweeps;         /* one-sided Jacobi sweeps over all updates                */
  int32_t max_bond;              /* largest bond dimension reached                          */
  int32_t hist_len;              /* chi_max + 1                                             */
  int64_t bond_hist[65];         /* bond_hist[d] = forward updates that left bond dim d     */
  double discarded_weight;       /* sum over trajectories of forward discarded weight       */
  double last_ms;                /* device time of the last call (CUDA events), ms          */
  double alg_flops;              /* algorithmic FP64 flops of the last evaluation: forward
                                    and costate updates, environments, overlaps (counted
                                    from the bond dimensions of every update; recomputation
                                    and extra Jacobi sweeps excluded)                       */
  double traj_ms;                /* device time of the trajectory-kernel launches since the
                                    previous tnrc_get_stats (CUDA events on the context's
                                    stream around each launch), ms                          */
  int64_t traj_launches;         /* number of those launches                                */
  int64_t restarts;              /* trajectories of the last evaluation whose forward history
                                    did not fit their CTA's region packed and that were redone
                                    with checkpoints (results are identical either way)     */
  int64_t phase_cycles[9];       /* SM cycles summed over warps per phase of the trajectory
                                    kernel (contraction, pivoted QR and the second QR,
                                    rank/truncate, split, environments, gradients, history
                                    copies, layer barriers, Jacobi sweeps); zero unless
                                    built with TNRC_PHASE_TIMERS                            */
  int64_t cap_truncations;       /* truncations of the last evaluation (forward and costate
                                    updates) whose cut the cap decided: more singular values
                                    exceeded the cutoff than chi_max keeps (Sec. II, D_max)  */
  double min_trunc_gap;          /* smallest (sigma_k - sigma_{k+1}) / sigma_1 over those cuts,
                                    k = chi_max: the relative distance between the last kept
                                    and the first dropped singular value.  Below 1e-10 the cut
                                    is a tie (the kept subspace is then decided by rounding,
                                    and two correct implementations may differ there); -1
                                    when the cap decided no cut                             */
} tnrc_stats;

/* Create a context on the current CUDA device, ordered on `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream).  inputs[P] are the initial
 * states |in_p>, targets[P] the targets |t_p>; both are brought to
 * normalised canonical form (chi_max and the cutoff applied) on the device.
 * Reserves all device memory the context will use.
 * Errors: TNRC_E_INVALID (bad sizes or NULLs), TNRC_E_NOMEM, TNRC_E_CUDA. */
tnrc_status tnrc_create(const tnrc_problem* problem, const tnrc_mps* inputs,
                        const tnrc_mps* targets, void* cuda_stream, tnrc_ctx** out);

/* Copy the controls u[K][C][N] (host, len = K*C*N doubles) to the device. */
tnrc_status tnrc_set_controls(tnrc_ctx* ctx, const double* u, int64_t len);

/* Draw J on the device from the counter-based SplitMix64 stream of `seed`:
 * dist 0 = uniform on [-scale, scale] (Sec. II), 1 = normal N(0, scale^2) by
 * Box-Muller.  Entry i of the flattened J[M][N-1] (or J[M][N-1][3]) uses
 * counter i (uniform) or counters 2i and 2i+1 (normal). */
tnrc_status tnrc_sample_noise(tnrc_ctx* ctx, uint64_t seed, int32_t dist, double scale);

/* Set J explicitly (host, len = M*(N-1)*crosstalk_terms doubles). */
tnrc_status tnrc_set_noise(tnrc_ctx* ctx, const double* J, int64_t len);

/* Copy the current J to the host (len = M*(N-1)*crosstalk_terms doubles).
 * Errors: TNRC_E_STATE if no noise was set or sampled yet. */
tnrc_status tnrc_get_noise(tnrc_ctx* ctx, double* J, int64_t len);

/* F (host scalar) and optionally per_traj[M][P] = |O_sp|^2 (host, may be NULL).
 * Errors: TNRC_E_STATE if controls or noise are missing. */
tnrc_status tnrc_fidelity(tnrc_ctx* ctx, double* F, double* per_traj);

/* F and grad[K][C][N] = dF/du (host) by the costate sweep (App. A).  The forward
 * layer states are kept packed at their actual bond dimensions for the sweep;
 * a trajectory whose history does not fit its CTA's region is redone with
 * checkpoints every checkpoint_every slices and recomputation (same results).
 * Errors: TNRC_E_STATE if controls or noise are missing; TNRC_E_NUMERIC if the
 * SVD did not converge or a non-finite value appeared. */
tnrc_status tnrc_fidelity_grad(tnrc_ctx* ctx, double* F, double* grad);

/* Overlaps O[M][P] (host, interleaved complex128) of the last evaluation. */
tnrc_status tnrc_get_overlaps(tnrc_ctx* ctx, double* overlaps, int64_t len);

/* Statistics of the last evaluation (synchronises the context's stream; the
 * trajectory-kernel timing accumulates over calls and is reset by this call). */
tnrc_status tnrc_get_stats(tnrc_ctx* ctx, tnrc_stats* stats);

/* Device-pointer forms for autograd and serving: stream-ordered on the
 * context's stream, asynchronous (no host synchronisation, no statistics
 * copy).  d_u is a device array [K][C][N]; d_F a device scalar; d_grad a
 * device array [K][C][N] (NULL for a forward-only evaluation); d_per_traj a
 * device array [M][P] or NULL.  Errors are detected at the next synchronous
 * call (tnrc_sync). */
tnrc_status tnrc_set_controls_dev(tnrc_ctx* ctx, const double* d_u);
tnrc_status tnrc_evaluate_dev(tnrc_ctx* ctx, double* d_F, double* d_grad, double* d_per_traj);
/* Run tnrc_evaluate_dev through CUDA graphs (enable = 1) or plain launches
 * (0, the default).  A graph is captured on the first call for each set of
 * output pointers (and each of "gates rebuilt" / "gates current") and replayed
 * on later calls; the trajectory-kernel timing of tnrc_get_stats does not
 * count graph replays.  The first evaluation of a context must not be inside
 * an application's own stream capture.  Errors: TNRC_E_INVALID when enabling
 * on a context created on the legacy default stream (it cannot be captured). */
tnrc_status tnrc_set_graphs(tnrc_ctx* ctx, int32_t enable);

/* F and grad[K][C][N] like tnrc_fidelity_grad, by the plain GPU path: one
 * trajectory at a time and one launch per step -- a launch per forward layer
 * whose CTAs (one warp each) take the layer's bonds, one for the overlap,
 * and per costate layer one for the environments and one for the bonds'
 * gradients and costate updates -- with every forward layer state kept as a
 * full slot.  The same device functions as the batched launch, so the
 * results are bitwise the same; it is the baseline the persistent batched
 * launch is measured against (no persistent CTAs, no batching across
 * trajectories, no CUDA graph).  Reserves its own device buffers on first
 * use ((L+1) full slots for L truncated layers, per-CTA scratch).  Errors as
 * tnrc_fidelity_grad, and TNRC_E_NOMEM. */
tnrc_status tnrc_fidelity_grad_plain(tnrc_ctx* ctx, double* F, double* grad);

/* Matrix shape of the trajectory kernel's SVDs: pairs = 1 (the default) lets
 * a warp take two small two-site updates at once, their pivoted QR and
 * Jacobi SVDs running on the two half-warps (when both thetas and both Phis
 * fit the warp's shared slab and no side exceeds 64), so the per-round
 * scalar work of the Jacobi is shared by two matrices; pairs = 0 gives every
 * SVD a whole warp.  Results agree within rounding (the sums run in another
 * lane arrangement); the plain path follows the same setting.  Captured
 * graphs are dropped when it changes.  The autotuner picks it per shape. */
tnrc_status tnrc_set_svd_shape(tnrc_ctx* ctx, int32_t pairs);

/* Order the context's later work on another stream (a cudaStream_t; NULL =
 * the legacy default stream, refused while graphs are on).  Waits for the
 * work already queued on the current stream first.  A serving loop uses it
 * to run one problem's requests at the priority each request deserves. */
tnrc_status tnrc_set_stream(tnrc_ctx* ctx, void* cuda_stream);

/* Launch the trajectory kernel pooled (enable = 1) or persistent (0, the
 * default).  Persistent: one CTA per resident slot, each taking trajectories
 * from a device counter until none are left -- the fastest form for one
 * evaluation alone, but its CTAs hold their SMs until the evaluation ends.
 * Pooled: one CTA per trajectory; a CTA takes one of the context's work
 * regions from a device pool while it runs (a bounded wait; TNRC_E_TIMEOUT if
 * it ever gave up) and hands it back when its trajectory is done, so the
 * block scheduler can start CTAs of other launches -- another context's
 * request on a higher-priority stream -- between trajectories.  Results are
 * bitwise the same in both forms.  Captured graphs are dropped when the form
 * changes.  Errors: TNRC_E_INVALID when the context's work regions cannot
 * cover the CTAs that could be resident at once (a memory-limited context). */
tnrc_status tnrc_set_pooled(tnrc_ctx* ctx, int32_t enable);

/* Synchronise the context's stream and report any device-side error flag. */
tnrc_status tnrc_sync(tnrc_ctx* ctx);

/* F and optionally per_traj[M][P] without allocating any device memory.
 *
 * For callers that cannot call cudaMalloc -- code inside a host runtime that
 * owns every device allocation, or a process that must not grow its device
 * footprint after start-up.  The paper has no counterpart: this is the same
 * evaluation as tnrc_create + tnrc_set_controls + tnrc_set_noise +
 * tnrc_fidelity (same kernels, same results), with every intermediate buffer
 * carved from one static device array of 32 MiB compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 *   problem, inputs[P], targets[P]: as for tnrc_create (host pointers);
 *   u[K][C][N], J[M][N-1] (x crosstalk_terms): host controls and noise;
 *   cuda_stream: cudaStream_t the work is ordered on (NULL = legacy default);
 *   F, per_traj (nullable): host outputs, written only on TNRC_OK.
 * Synchronous at return.  Returns TNRC_E_TOO_LARGE when the problem's buffers
 * (gate table, canonical states, one working state per CTA and its scratch)
 * do not fit the 32 MiB array or an input bond dimension exceeds 64.  The
 * array is shared by every call and keeps the last call's contents (each call
 * clears what must start at zero); calls whose device work overlaps race on
 * it and must be serialised.  Every call looks up the array's device address
 * on the current device and synchronises its stream before returning.  With
 * CUDA's lazy module loading (the default) the array is placed on a device at
 * the first call there (or at library load with CUDA_MODULE_LOADING=EAGER), so
 * a caller that must not grow its device footprint later makes one small
 * call at start-up; after that, calls allocate nothing.  Problems are
 * validated by the same rules as tnrc_create (TNRC_E_INVALID). */
tnrc_status tnrc_fidelity_static(const tnrc_problem* problem, const tnrc_mps* inputs,
                                 const tnrc_mps* targets, const double* u, const double* J,
                                 void* cuda_stream, double* F, double* per_traj);

/* Bytes of device memory tnrc_create would reserve for this problem (0 on bad input). */
size_t tnrc_footprint(const tnrc_problem* problem);

/* Release every resource of the context (NULL is accepted). */
void tnrc_destroy(tnrc_ctx* ctx);

/* Measure the current device's FP64 FMA throughput (GFLOP/s): 8 independent
 * FMA chains per thread on 4 CTAs x 256 threads per SM, best of 4 timed
 * launches after a warm-up, on the legacy default stream.  `scratch` is a
 * device buffer of at least 4 * SMs * 256 doubles (written, not read).  The
 * roofline denominator of the trajectory kernel, which is bound by FP64
 * arithmetic (the paper has no counterpart; it quotes no hardware). */
tnrc_status tnrc_measure_fp64_peak(void* scratch, size_t scratch_bytes, double* gflops);

/* Measure the current device's FP64 tensor-core (DMMA, m8n8k4) throughput in
 * GFLOP/s: 4 independent multiply-accumulate chains per warp on 4 CTAs x 256
 * threads per SM, best of 4 timed launches after a warm-up, on the legacy
 * default stream; `scratch` as above.  It tells whether the trajectory
 * kernel's contractions would gain from the FP64 tensor path (the paper has
 * no counterpart; it quotes no hardware). */
tnrc_status tnrc_measure_dmma_peak(void* scratch, size_t scratch_bytes, double* gflops);

/* After TNRC_E_CUDA: which CUDA call failed and why ("" otherwise).  The
 * string lives as long as the context. */
const char* tnrc_last_error(const tnrc_ctx* ctx);

/* Human-readable name of a status code. */
const char* tnrc_status_string(tnrc_status status);

#ifdef __cplusplus
}
#endif
#endif /* TNRC_H */
