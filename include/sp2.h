/*
 * sp2.h -- C ABI of the GB300 SP2 density-matrix / response / susceptibility
 * library (libsp2.so).
 *
 * The operations follow A. M. N. Niklasson et al., "Susceptibility Formulation
 * of Density Matrix Perturbation Theory" (arXiv 2409.17033):
 *
 *   sp2_density        Eq. DM0 (Sec. II): D = theta(mu I - H) by the SP2
 *                      recursive Fermi-operator expansion, Tr[D] = N_occ.
 *   sp2_response       Eq. DMPert (Appendix; Eq. DM1 merged with Eq. DM0):
 *                      first-order density-matrix responses D1_k to a batch
 *                      of Hamiltonian perturbations H1_k.
 *   sp2_susceptibility Eq. DMSuscept (Appendix; Eq. DM3 merged with Eq. DM0),
 *                      forward, or Eq. DM2 (Sec. IV.A), backward/adjoint over
 *                      the stored or recomputed X_n: chi^A_l of a batch of
 *                      observables A_l, chi^A_ij = d Tr[A D] / d H_ij (Eq. Suscept).
 *   sp2_adjoint        Eq. DM2 on the X_n history kept by the handle's last
 *                      sp2_density call (the backward pass of an autograd
 *                      wrapper: grad_H = chi^G for the incoming gradient G).
 *   response_contract  a1[l,k] = Tr[P_l Q_k] (Eqs. expectation, direct, dual):
 *                      Tr[chi^A_l H1_k] or Tr[A_l D1_k], accumulated in FP64.
 *
 * Conventions shared by every call
 * --------------------------------
 * Matrices are dense, square N x N, row-major and contiguous; a batch of B
 * matrices is B*N*N contiguous elements. H, H1_k, A_l must be symmetric (the
 * paper assumes S = I and symmetric operators, Sec. I); symmetry is not
 * checked. The element type of every caller matrix is given by `dtype`
 * (SP2_F64 = double, SP2_F32 = float); `out` of response_contract is always
 * double.
 *
 * Pointers may be device memory (cudaMalloc, torch tensors) or host memory
 * (pageable or pinned); host buffers are staged through handle-owned device
 * memory with copies on the handle's stream. The library never frees or keeps
 * caller memory.
 *
 * Asynchrony. All device work is enqueued on the handle's stream. The SP2
 * step loop never drains that stream: the host reads the branch/stop state
 * from pinned snapshots at most 8 steps behind the step it enqueues (those
 * steps become no-ops on the device once the recursion has stopped), so the
 * stop, M and the kept iterate are known when sp2_density, sp2_response and
 * sp2_susceptibility return, while the remaining device work (the last steps,
 * the adjoint of a backward susceptibility, output copies) may still run.
 *   - info == NULL and every output in device memory: the call returns without
 *     waiting; outputs are valid once the stream has reached them, and
 *     sp2_synchronize(h, info) waits, reports the call's final status and fills
 *     its info.
 *   - info != NULL, or an output in host memory: the call waits for its work
 *     and returns the final status with info filled (synchronous use).
 * sp2_adjoint behaves the same way. sp2_fermi, sp2_nonorth_susceptibility,
 * sp2_scf_response and response_contract always return after their work is
 * done. Statuses known when a call returns (bad arguments, ENOCONV, a NaN
 * found by the stop test, a timed-out wait seen by the step loop) are returned
 * at once; a timed-out wait in later work of the call (the adjoint) is
 * reported by sp2_synchronize.
 *
 * Internal working storage (padded copies, X ping-pong buffers, split planes,
 * the X_n checkpoints of the adjoint, reduction partials) is owned by the
 * handle, grows on demand up to `workspace_limit_bytes` (0 = no limit) and is
 * freed by sp2_destroy.
 *
 * Return value: an sp2_status. On failure nothing is guaranteed about the
 * outputs; sp2_last_error(h) gives a message (handle-owned string, valid
 * until the next call on that handle). No exception crosses the ABI.
 * A handle is not thread-safe: one host thread at a time.
 */
#ifndef SP2_H
#define SP2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SP2_MAX_ITER 256
#define SP2_CKPT_AUTO (-1)  /* sp2_opts.ckpt_k: choose k from free device memory */

typedef enum {
  SP2_OK = 0,
  SP2_EINVAL = 1,      /* bad argument (null pointer, negative size, bad enum, N_occ out of [0,N]) */
  SP2_ENOMEM = 2,      /* device allocation failed or workspace limit exceeded */
  SP2_ENOCONV = 3,     /* max_iter steps without meeting the stop rule (outputs hold the last iterate) */
  SP2_ENONFINITE = 4,  /* NaN/Inf in the spectral bounds or traces (non-finite input) */
  SP2_ETIMEOUT = 5,    /* a device-side wait hit its time limit; the kernel bailed out */
  SP2_ECUDA = 6,       /* a CUDA runtime/driver call failed (message has the CUDA error) */
  SP2_ENOTIMPL = 7,    /* combination not implemented */
  SP2_ENOSTATE = 8     /* sp2_adjoint without a kept X_n history on this handle */
} sp2_status;

typedef enum { SP2_F64 = 0, SP2_F32 = 1 } sp2_dtype;

/* Arithmetic of the matrix products (Sec. VI.B).
 *   SP2_MODE_FP64    plain FP64 (CUDA-core DFMA).
 *   SP2_MODE_FP32    plain FP32 (CUDA-core FFMA): the paper's "GPU FP32" form.
 *   SP2_MODE_BF16X2  Eq. doubleHalf / Eq. MixPrecMult with bfloat16 hi/lo planes:
 *                    three tensor-core products (hi*hi + hi*lo + lo*hi, lo*lo
 *                    dropped, Eq. mults), FP32 accumulation, FP32 master copy.
 *   SP2_MODE_FP16X2  the same with fp16 planes, the paper's own format: the lo
 *                    plane holds the residual times 2^11 and is accumulated
 *                    separately; response matrices carry a per-matrix
 *                    power-of-two scale so that no plane entry exceeds 2^14.
 *   SP2_MODE_BF16X3  three bfloat16 planes hi + mid + lo (exact for FP32 values)
 *                    and six tensor-core products keeping every term down to
 *                    2^-16 relative (hi*hi; hi*mid, mid*hi; hi*lo, mid*mid,
 *                    lo*hi): the multi-split extension of Eq. MixPrecMult
 *                    that Sec. VI.C names for tunable accuracy; twice the
 *                    tensor work of the two-plane modes, no scaling.
 *   SP2_MODE_BF16_TAIL  the bfloat16-bulk / split-tail form of Sec. VI.B (tensor-
 *                    core results as the start of higher-precision work in the
 *                    last iterations): SP2_MODE_BF16X2 with the split-tail option
 *                    (sp2_opts.tail_f, below) on; tail_f = 0 takes
 *                    SP2_DEFAULT_TAIL_F. The calls run and report it as
 *                    SP2_MODE_BF16X2 with that tail_f. Its density error is set by
 *                    the bulk's bfloat16 rounding times the condition number (the
 *                    split tail restores idempotency, not the subspace).
 */
typedef enum {
  SP2_MODE_FP64 = 0,
  SP2_MODE_FP32 = 1,
  SP2_MODE_BF16X2 = 2,
  SP2_MODE_FP16X2 = 3,
  SP2_MODE_BF16X3 = 4,
  SP2_MODE_BF16_TAIL = 5
} sp2_mode;

/* tail_f of SP2_MODE_BF16_TAIL when the caller leaves it at 0 */
#define SP2_DEFAULT_TAIL_F 1.0

typedef struct {
  int mode;            /* sp2_mode */
  double idem_tol;     /* stop when |e_{n+1}| <= idem_tol; <= 0 disables this test.
                          e_n = Tr[X_n] - ||X_n||_F^2 is the idempotency error (Sec. II). */
  double floor_gate;   /* precision-floor stop on f_n = ||X_n - X_n^2||_F^2 (< 0 selects the
                          default 0.03, 0 disables). After step n it fires when steps n-2 and
                          n-1 took opposite branches, f_{n-2} <= floor_gate and f_n >= f_{n-2},
                          or when the smallest f so far is <= floor_gate and none of the last
                          4 steps went below it. In exact arithmetic neither happens once
                          f <= 0.03 (every eigenvalue is within 1/4 of 0 or 1 and a pair of
                          opposite branches maps a distance d to at most 4 d^2). The result
                          is then the iterate X_n (n >= 2, f_n <= floor_gate) with the
                          smallest f_n, so M = n - 1: past the floor f cycles with rounding,
                          and the near-gap response terms follow it. */
  int max_iter;        /* cap on SP2 steps M (1..SP2_MAX_ITER; 0 = default 100) */
  int min_iter;        /* no stop test before this step (default 4 when < 0) */
  int fixed_m;         /* > 0: take exactly fixed_m steps with the branches in sigma_in */
  const int8_t* sigma_in; /* host array of fixed_m branch signs (+1 square, -1 2X-X^2) */
  double eps_min;      /* if eps_min < eps_max: spectral bounds to use instead of the */
  double eps_max;      /* Gershgorin estimate (Sec. II: alpha, beta from eps_min/eps_max) */
  int ckpt_k;          /* sp2_density keep_history / backward chi: keep X_n every ckpt_k
                          steps and recompute the rest per segment (0 = default 4). 1 keeps
                          every X_n (split modes: its hi/lo planes) and recomputes nothing.
                          SP2_CKPT_AUTO: the smallest k whose history of max_iter steps fits
                          in free device memory (and the workspace limit) beside the working
                          set, so X_n is recomputed only when the history outgrows HBM. */
  int keep_history;    /* sp2_density: keep the X_n checkpoints for a later sp2_adjoint */
  int time_kernels;    /* 1: bracket every product-kernel launch with CUDA events on the
                          handle's stream and report their summed duration in sp2_info */
  double tail_f;       /* split modes, > 0: split-tail arithmetic (the mixed-precision use the
                          paper suggests in Sec. VI.B: low precision in the bulk of the
                          iterations, higher precision in the last ones). Step n uses the hi
                          planes alone (one 16-bit product, FP32 accumulation) while
                          f = ||X - X^2||_F^2 of the last measured iterate exceeds tail_f, and
                          the split products from the first step where it does not on (the
                          decision is made on the device; the adjoint follows the same steps).
                          With SP2_MODE_BF16X2 this is the bfloat16 bulk / split tail form.
                          0 (default): split products in every step. */
  int block_sparse;    /* sp2_density, split modes, CTA-pair products (the default), N <= 65536:
                          != 0 runs Eq. DM0 in thresholded block-sparse algebra (Sec. II's
                          remark on thresholded sparse matrix products). The iterates are cut
                          into 256 x 256 blocks; after X_1 and after every step, each
                          off-diagonal block whose Frobenius norm is <= block_tau is set to
                          zero (diagonal blocks always stay), and a square forms only the
                          blocks (I, J) reachable through kept blocks (I, K), (K, J), over those
                          K alone. block_tau = 0 drops only blocks that are exactly zero (the
                          dense result, bit for bit, with the zero blocks skipped). The stop
                          test adds one floor rule: from f <= 1e-4, two steps of opposite
                          branches that cut f by less than half mark the threshold's floor.
                          Storage stays dense. 0 (default): the dense recursion. The other
                          entry points reject != 0. */
  double block_tau;    /* the block threshold (>= 0, finite) when block_sparse != 0 */
} sp2_opts;

typedef struct {
  int M;               /* SP2 steps taken */
  int converged;       /* 1 if a stop rule fired (or fixed_m given) */
  double alpha, beta;  /* X_1 = alpha I + beta H */
  double eps_min, eps_max;
  double trace;        /* Tr[D] in FP64 */
  double idem_err;     /* e of D = X_{M+1} */
  int8_t sigma[SP2_MAX_ITER];         /* sigma_1..sigma_M */
  double errors[SP2_MAX_ITER + 1];    /* e of X_1..X_{M+1} */
  double idem_fro[SP2_MAX_ITER];      /* f = ||X_n - X_n^2||_F^2 of X_1..X_M */
  int64_t n_gemm_launches;            /* product-kernel launches that did work */
  double executed_flops;              /* tensor/FMA flops issued by the product kernels (FMA = 2) */
  double algorithmic_flops;           /* flops the products need by definition: the upper
                                         triangle (with diagonal) of X^2, all of Y X, on the
                                         caller's N (not the padding), x3 for the split form */
  int64_t kernel_launches;            /* every kernel this call launched (no-op launches included) */
  double product_ms;                  /* time_kernels: summed event time of the product launches
                                         that did work, else 0 */
  int64_t product_launches_timed;
  int ckpt_k;                         /* checkpoint interval the call used (backward chi and
                                         keep_history; SP2_CKPT_AUTO resolved), else 0 */
  int refine_iter;                    /* sp2_scf_response: first iteration (0-based) computed
                                         in refine_mode, -1 if none; sp2_nonorth_susceptibility:
                                         Newton-Schulz iterations of S^(-1/2) */
  int tail_single_steps;              /* split-tail mode: steps 1..M that used the hi planes
                                         alone (executed_flops and algorithmic_flops count
                                         split products for every step) */
  double block_fill;                  /* block-sparse recursion (block_sparse): mean over steps
                                         1..M of the share of the upper 256 x 256 blocks each
                                         square formed (1 = dense); executed_flops and
                                         algorithmic_flops then count the K blocks the squares
                                         ran */
} sp2_info;

typedef struct sp2_handle_s* sp2_handle_t;

/* Fill *opts with defaults (mode FP32, idem_tol 0, floor_gate 0.03, max_iter 100, min_iter 4,
 * ckpt_k 4). */
void sp2_default_opts(sp2_opts* opts);

/* Create a handle bound to the current CUDA device and `cuda_stream` (a
 * cudaStream_t; NULL = legacy default stream). Returns SP2_EINVAL for a null
 * out-pointer, SP2_ECUDA if no device is usable. */
int sp2_create(sp2_handle_t* out, void* cuda_stream, size_t workspace_limit_bytes);
int sp2_destroy(sp2_handle_t h);
int sp2_set_stream(sp2_handle_t h, void* cuda_stream);
const char* sp2_last_error(sp2_handle_t h);
/* Bytes of device memory the handle currently holds. */
size_t sp2_workspace_bytes(sp2_handle_t h);

/* Launch settings of the tensor-core product kernel (not part of the arithmetic).
 *   SP2_OPTION_WAIT_LIMIT_NS  limit of every bounded device wait, in ns (default
 *                             2e9). When a wait runs out the kernel raises an abort
 *                             flag, drains its own copies and tensor-core work,
 *                             frees its tensor memory and returns; the call then
 *                             returns SP2_ETIMEOUT and the handle stays usable.
 *   SP2_OPTION_WITHHOLD_LOAD  test hook for that path: != 0 makes the first
 *                             operand load of the first CTA of every product
 *                             launch never be issued, so the wait for it runs out
 *                             (use with a short wait limit). Default 0.
 *   SP2_OPTION_FUSED_RESPONSE != 0: each response step of the split modes is one
 *                             tensor-core launch over the upper tiles that forms
 *                             Y X + X Y as [Y | X] . [X ; Y] and applies the branch
 *                             update in its epilogue (no Y X buffer, no separate
 *                             transpose-add pass); 0 (default): Y X, then the
 *                             transpose-add kernel. Same arithmetic up to rounding
 *                             order.
 *   SP2_OPTION_PAIR_TILES     != 0 (default): the split modes' products run on
 *                             pairs of SMs (a thread-block cluster of two), each
 *                             pair computing 256 x 256 output tiles with one
 *                             tensor-core instruction stream over both SMs; 0: one
 *                             SM per 128 x 256 tile. Same arithmetic and summation
 *                             order, hence the same results.
 * Returns SP2_EINVAL for an unknown option or a value out of range. */
typedef enum {
  SP2_OPTION_WAIT_LIMIT_NS = 0,
  SP2_OPTION_WITHHOLD_LOAD = 1,
  SP2_OPTION_FUSED_RESPONSE = 2,
  SP2_OPTION_PAIR_TILES = 3
} sp2_option;
int sp2_set_option(sp2_handle_t h, int option, int64_t value);

/* Eq. DM0. H: N x N input. nocc: N_occ in [0, N]. D: N x N output.
 * info (nullable, host): M, branch sequence, errors, alpha/beta. */
int sp2_density(sp2_handle_t h, const void* H, int64_t N, int dtype, double nocc,
                const sp2_opts* opts, void* D, sp2_info* info);

/* Eq. DMPert: K first-order responses D1_k (K x N x N) to H1_k. If
 * h1_diag_only != 0, H1 holds only the K diagonals (K x N), i.e.
 * H1_k = diag(H1[k, :]). D (nullable) receives D^(0). K = 0 is allowed. */
int sp2_response(sp2_handle_t h, const void* H, int64_t N, int dtype, double nocc,
                 const void* H1, int64_t K, int h1_diag_only, const sp2_opts* opts,
                 void* D, void* D1, sp2_info* info);

/* Susceptibilities chi^A_l (L x N x N) of L observables A_l.
 * direction 0: forward, Eq. DMSuscept (X_n generated on the fly, nothing stored).
 * direction 1: backward, Eq. DM2, X_n kept every opts->ckpt_k steps and the
 *              rest recomputed segment by segment.
 * a_diag_only != 0: A holds only the L diagonals (L x N). D (nullable) receives D^(0). */
int sp2_susceptibility(sp2_handle_t h, const void* H, int64_t N, int dtype, double nocc,
                       const void* A, int64_t L, int a_diag_only, int direction,
                       const sp2_opts* opts, void* D, void* chi, sp2_info* info);

/* Eq. DM2 against the X_n history kept by the last sp2_density(keep_history=1)
 * on this handle: G (N x N, symmetric, dtype of that call) -> grad (N x N) with
 * grad = d Tr[G D] / d H. SP2_ENOSTATE if no history is kept or N differs. */
int sp2_adjoint(sp2_handle_t h, const void* G, int64_t N, int dtype, void* grad, sp2_info* info);

/* Release a kept X_n history (device memory) without destroying the handle. */
int sp2_release_history(sp2_handle_t h);

/* Wait for the handle's stream and complete the last call that returned
 * without waiting (see "Asynchrony" above): returns that call's final status
 * (e.g. SP2_ETIMEOUT for a timed-out wait in its adjoint) and fills *info
 * (nullable) as the synchronous form of the call would have. With no such call
 * pending it waits for the stream, zeroes *info and returns SP2_OK. Only the
 * most recent call is reported: a call made before the previous one was
 * synchronised discards the previous one's report (its work still runs). */
int sp2_synchronize(sp2_handle_t h, sp2_info* info);

/* Finite electronic temperature (Sec. V.B): the Fermi-Dirac density matrix
 *     D = f(H) = (exp((H - mu I) / kT) + I)^(-1)
 * and the first-order responses D1_k = d f(H + lambda B_k) / d lambda, which
 * are the finite-temperature susceptibilities chi^A when B_k = A (Eq.
 * Suscept_Der). canonical != 0 adds the chemical-potential response mu_1
 * chosen so that Tr[D1_k] = 0 (the mu_1 rule stated with Eq. CP_SCF);
 * canonical = 0 gives the grand-canonical response at fixed mu.
 *
 * The paper cites the recursion without printing it; the one implemented is
 * the odds-squaring recursion f(2x) = f(x)^2 / (f(x)^2 + (1 - f(x))^2), written
 * for delta = f - 1/2:
 *     delta_0 = -(1 / (kT 2^(n+2))) (H - mu I),
 *     delta_{j+1} = 2 delta_j (I + 4 delta_j^2)^(-1),  j < n,   D = I/2 + delta_n,
 * with n = n_doublings, the inverse by Newton-Schulz iterations whose count
 * follows from a spectral bound of delta_j, and the responses by the chain
 * rule of each step over the stored delta_j. The result is the Fermi
 * function of H up to a log-odds error of 2 (x/2)^3 / (3 4^n), x = (e - mu)/kT.
 * Requires |e - mu| / (kT 2^(n+2)) < 1/2 over the Gershgorin bounds of H
 * (SP2_EINVAL otherwise: raise n_doublings).
 * H: N x N. B: K x N x N, or K x N diagonals when b_diag_only != 0; K = 0 is
 * allowed. opts->mode selects the arithmetic (all four modes). D (nullable):
 * N x N. D1: K x N x N. info->M = n_doublings. */
int sp2_fermi(sp2_handle_t h, const void* H, int64_t N, int dtype, double mu, double kT,
              const void* B, int64_t K, int b_diag_only, int canonical, int n_doublings,
              const sp2_opts* opts, void* D, void* D1, sp2_info* info);

/* Non-orthonormal basis (Sec. V.A): H, S (overlap, symmetric positive definite)
 * and the observable A in the atomic-orbital representation, N x N (dtype,
 * device or host). With the Loewdin factor Z = S^(-1/2) (coupled Newton-Schulz
 * iteration on the device), H^perp = Z H Z, A^perp = Z A Z, D^perp from Eq. DM0,
 * chi^perp from Eq. DM2, and D = Z D^perp Z. Outputs (N x N, dtype):
 *   D    the density matrix in the atomic-orbital representation;
 *   W_H  = Z chi^perp Z;
 *   W_S  = -sym(S^-1 H W_H) - sym(S^-1 A D), sym(M) = (M + M^T) / 2;
 *   Z    (nullable) the Loewdin factor.
 * The derivative of a = Tr[A D] along any basis-set dependent perturbation
 * (Eq. NonOrthDer with Z_tau = -S^-1 S_tau Z / 2, dual form Tr[A^perp D^perp_tau]
 * = Tr[chi^perp H^perp_tau]) is then three contractions,
 *   a_tau = Tr[A_tau D] + Tr[W_H H_tau] + Tr[W_S S_tau],
 * e.g. with response_contract. opts as for sp2_susceptibility (fixed_m is not
 * accepted); info is that of the SP2 / susceptibility solve on H^perp with the
 * product counts of the whole call, and info->refine_iter holds the number of
 * Newton-Schulz iterations. SP2_EINVAL for an overlap whose Gershgorin bound
 * is not positive, SP2_ENOCONV if the inverse square root does not converge. */
int sp2_nonorth_susceptibility(sp2_handle_t h, const void* H, const void* S, int64_t N, int dtype,
                               double nocc, const void* A, const sp2_opts* opts, void* D,
                               void* W_H, void* W_S, void* Z, sp2_info* info);

/* Self-consistent first-order response (Appendix, Eq. DM_CP_SCF; its dual is
 * Eq. CP_SCF) with a site-charge interaction: for each of F external site
 * potentials V_ext (F x n_sites), find site charges q with
 *     q = q_out(q),  q_out(q) = site charges of D1[H1 = diag(u (x) 1_norb)],
 *     u = V_ext + K q  (K: n_sites x n_sites),  q_a = sum_{mu in site a} D1_{mu mu},
 * D1 being the zero-temperature response of Eq. DM1 (merged form, Eq. DMPert)
 * to the site-diagonal perturbation u. N = n_sites * norb; orbitals of site a
 * are a*norb .. a*norb+norb-1.
 * Mixers: linear (the paper's constant c_mix = alpha), Anderson over the last
 * `history` iterates (the "more advanced SCF acceleration" the Appendix
 * mentions), or a learned correction to linear mixing,
 * q <- q + alpha r + ||r|| MLP(r / ||r||), r = q_out - q, with
 * y = W2 relu(W1 x) (no biases; W1: hidden x n_sites, W2: n_sites x hidden,
 * device FP32; bf16_infer rounds weights and activations to bfloat16), or
 * Anderson with that learned step as its preconditioner (SP2_MIX_ANDERSON_MLP).
 * The residual judging convergence is the plain method's:
 * ||q_out(q) - q||_2 / ||q_out(0)||_2 over all fields, stopping at <= tol.
 * K, V_ext and q (F x n_sites out, the last iterate) are double, device or
 * host. residuals: host array of max_iter doubles (nullable); iterations:
 * host int. traj_r / traj_q (nullable, device doubles of max_iter x F x
 * n_sites): residual and iterate of every iteration (training data). */
typedef enum {
  SP2_MIX_LINEAR = 0,
  SP2_MIX_ANDERSON = 1,
  SP2_MIX_MLP = 2,
  SP2_MIX_ANDERSON_MLP = 3  /* Anderson with the learned step as its preconditioner:
                               q <- sum_i c_i (q_i + P(r_i)), P(r) = alpha r + ||r|| MLP(r/||r||) */
} sp2_mixer;

typedef struct {
  int mixer;            /* sp2_mixer */
  double alpha;         /* linear mixing parameter; Anderson's damping of the residual */
  int history;          /* Anderson history length (1..32) */
  double tol;           /* relative residual tolerance */
  int max_iter;         /* SCF iteration cap */
  const float* W1;      /* MLP weights (device) for SP2_MIX_MLP */
  const float* W2;
  int hidden;           /* MLP width */
  int bf16_infer;       /* 1: bfloat16 operands in inference */
  int refine_mode;      /* sp2_mode of the responses after the switch below */
  double refine_below;  /* > 0: once the residual is <= refine_below, or has not reached a
                           new minimum for 3 iterations, the remaining iterations compute
                           the responses in refine_mode, and Anderson restarts its history.
                           The SP2 polynomial (branches, M, bounds) of the first iterations
                           is kept, except for SP2_MODE_FP64, whose own SP2 run fixes it again
                           (to its tighter floor). 0 = never switch. Lets split-precision
                           responses do the bulk of the iterations and FP32 / FP64 ones go
                           below their rounding floor. */
  double kT;            /* > 0: finite-temperature responses (Sec. V.B recursion, as in
                           sp2_fermi) at chemical potential mu; 0: zero temperature (Eq. DM1) */
  double mu;
  int n_doublings;      /* finite T: doublings of the recursion (0 = 20) */
  int canonical;        /* finite T: 1 = canonical responses (mu_1 with Tr[D1] = 0) */
} sp2_scf_opts;

int sp2_scf_response(sp2_handle_t h, const void* H, int64_t N, int dtype, double nocc, int norb,
                     const double* Ksite, const double* Vext, int64_t F, const sp2_scf_opts* so,
                     const sp2_opts* opts, double* q, double* residuals, int* iterations,
                     double* traj_r, double* traj_q, sp2_info* info);

/* Learned preconditioner kernels (FP32 training, bf16 or FP32 inference).
 * The map is y = W2 relu(W1 x) for x of length d_in, W1: d_h x d_in,
 * W2: d_in x d_h, all row-major device FP32; X, T, Y are P x d_in.
 * The paper has no learned part; these serve the SCF mixer above. */
int sp2_mlp_forward(sp2_handle_t h, const float* W1, const float* W2, int d_in, int d_h,
                    const float* X, int64_t P, float* Y, int bf16);
/* Mean squared error L = sum (Y - T)^2 / P and its gradients dW1, dW2
 * (device FP32); *loss is a host double. */
int sp2_mlp_loss_grad(sp2_handle_t h, const float* W1, const float* W2, int d_in, int d_h,
                      const float* X, const float* T, int64_t P, double* loss, float* dW1,
                      float* dW2);
/* `steps` full-batch Adam steps (beta 0.9 / 0.999, eps 1e-8) on (X, T),
 * updating W1, W2 in place; loss_hist (host, nullable) gets each step's loss. */
int sp2_mlp_train(sp2_handle_t h, float* W1, float* W2, int d_in, int d_h, const float* X,
                  const float* T, int64_t P, int steps, double lr, double* loss_hist);

/* out[l*K + k] = sum_ij P_l[i,j] * Q_k[i,j] (= Tr[P_l Q_k] for symmetric P_l or Q_k),
 * accumulated in FP64. P: L x N x N. Q: K x N x N, or K x N diagonals when
 * q_diag_only != 0 (then out = sum_i P_l[i,i] Q_k[i]). out: L*K doubles
 * (device or host). L or K = 0 is allowed (nothing written). */
int response_contract(sp2_handle_t h, const void* P, int64_t L, const void* Q, int64_t K,
                      int64_t N, int dtype, int q_diag_only, double* out);

/* response_contract_noalloc: the same contraction as response_contract for
 * callers that cannot allocate device memory -- code whose device memory is
 * owned entirely by another allocator, or which must not pay for the device
 * synchronisation that cudaMalloc/cudaFree can imply -- and that therefore
 * cannot create a handle. The paper has no counterpart to this entry point.
 *
 * Nothing is allocated or freed by any call: the reduction partials live in
 * one file-scope device array of 2^17 doubles (1 MiB), which every GPU that
 * loads libsp2.so holds until the process exits. The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress, with that
 * device current) and caches it; make that first call before any stream
 * capture begins. P, Q and out must be device memory of the current device
 * (host pointers and memory of another GPU are rejected);
 * out[l*K + k] = sum_ij P_l[i,j] Q_k[i,j] as in response_contract.
 * The work is enqueued on `cuda_stream` (a cudaStream_t, NULL = legacy
 * default stream) and the call returns without waiting: out is valid once
 * the stream has reached it. All calls share the one partial-sum array,
 * which keeps the last call's contents; every partial a call reads is written
 * by that same call first, so nothing needs clearing, but calls whose work
 * overlaps on the GPU (other streams, other host threads) race on the array
 * and must be ordered by the caller.
 * Returns SP2_EINVAL for negative sizes, a bad dtype, null, host or
 * other-GPU pointers, or L * K > 65535; SP2_ECUDA if a CUDA call fails. */
int response_contract_noalloc(const void* P, int64_t L, const void* Q, int64_t K, int64_t N,
                              int dtype, int q_diag_only, double* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SP2_H */
