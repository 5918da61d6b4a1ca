/* Learned warm start of the MS-GFEM local eigensolver: C ABI.
 *
 * The paper has no learned component.  Its conclusion (Sec. 6) suggests
 * reusing local spaces computed once for new inputs; this part goes one step
 * further: a small multilayer perceptron maps a subdomain's ply-angle
 * perturbation field to a start block for the block Krylov eigensolver of
 * msgfem_local_spaces.  The eigensolver still iterates to the same tolerance;
 * a poor start block only costs iterations, and the random start block stays
 * the fallback.
 *
 * Network: layer widths s_0 .. s_L; hidden layers h = tanh(W h_prev + b), the
 * output layer is linear; loss = mean of (y - t)^2 over all batch x s_L
 * entries; Adam (Kingma and Ba, ICLR 2015, Algorithm 1).  All network
 * arithmetic is FP32.  Parameters are one flat vector W_1 [s_1][s_0], b_1
 * [s_1], W_2 [s_2][s_1], b_2, ... (row-major weights).  Batches are row-major
 * [batch][width] device arrays.
 *
 * Errors: every call returns an msgfem_status (include/msgfem.h); EINVAL for
 * NULL handles, non-positive sizes or a batch above the capacity given at
 * creation; ECUDA for a failed CUDA call.  Calls on one handle are not
 * thread-safe; work is issued on the handle's stream.
 */
#ifndef MSGFEM_WARM_H
#define MSGFEM_WARM_H

#include "msgfem.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct msgfem_net* msgfem_net_h;

/* Create a network with n_sizes layer widths (n_sizes >= 2, each >= 1) for
 * batches of at most max_batch rows.  init_params (host, param_count floats)
 * may be NULL (all zero).  stream: cudaStream_t or NULL.  The handle owns all
 * device memory (parameters, Adam moments, activations). */
msgfem_status msgfem_net_create(int n_sizes, const int* sizes, int max_batch, const float* init_params,
                                void* stream, msgfem_net_h* out);

/* Number of parameters (floats) of the network. */
long long msgfem_net_param_count(msgfem_net_h net);

/* Copy the parameters to / from a host array of msgfem_net_param_count floats
 * (synchronous).  set_params also resets the Adam moments and step count. */
msgfem_status msgfem_net_get_params(msgfem_net_h net, float* host_out);
msgfem_status msgfem_net_set_params(msgfem_net_h net, const float* host_in);

/* Y [batch][s_L] = f(X [batch][s_0]); device pointers, asynchronous. */
msgfem_status msgfem_net_forward(msgfem_net_h net, const float* X, int batch, float* Y);

/* Loss and gradient at the current parameters for targets T [batch][s_L]
 * (device); grad_out (host, param_count floats) and loss_out (host) may be
 * NULL.  Synchronous when either output is given. */
msgfem_status msgfem_net_gradient(msgfem_net_h net, const float* X, const float* T, int batch,
                                  float* grad_out, double* loss_out);

/* One Adam step on the batch (forward, backward, update).  loss_out (host,
 * loss before the update) may be NULL, which keeps the call asynchronous. */
msgfem_status msgfem_net_adam_step(msgfem_net_h net, const float* X, const float* T, int batch, float lr,
                                   float beta1, float beta2, float eps, double* loss_out);

void msgfem_net_destroy(msgfem_net_h net);

/* Per-subdomain features for the network: the perturbation field dtheta
 * (device, one double per element in the element order of
 * msgfem_plies.elem_angle_deg, degrees) on the elements of Omega*_j, times
 * scale, in the element order (i, j, k) of the Omega* box (k fastest).
 * feat (device, N x ld floats, row j for subdomain j) receives them; entries
 * of row j beyond subdomain j's element count are zero.  *nfeat_out (may be
 * NULL) receives the largest element count over the subdomains; EINVAL if ld
 * is smaller than that.  feat = NULL only queries *nfeat_out.  Asynchronous
 * on the msgfem handle's stream. */
msgfem_status msgfem_warm_features(msgfem_h h, const double* dtheta, float scale, float* feat, int ld,
                                   int* nfeat_out);

/* Size of the interface (B2) block of subdomain j (rows of its start block)
 * and the number of wanted non-rigid eigenpairs nw_j = n_loc - 6 for a
 * floating subdomain, n_loc otherwise (subdomain j's n_loc in the last
 * msgfem_local_spaces or msgfem_local_spaces_var call, or the argument when
 * > 0). */
msgfem_status msgfem_warm_sizes(msgfem_h h, int j, int n_loc, int* n2_out, int* nw_out);

/* After msgfem_local_spaces: the wanted non-rigid eigenvectors of subdomain j
 * restricted to its B2 rows (full-layout row order), as out [n2_j][ld] FP32
 * (device; columns nw_j .. ld - 1 are zeroed).  With ref (device,
 * [n2_j][ld], first nw_j columns used) the block is rotated by the
 * orthogonal Q minimising ||X Q - ref||_F (orthogonal Procrustes), which
 * removes the sign and rotation freedom of the eigenvectors.  ld >= KB (8).
 * Asynchronous.  Errors: ESTATE before msgfem_local_spaces. */
msgfem_status msgfem_warm_targets(msgfem_h h, int j, const float* ref, float* out, int ld);

/* Start block of subdomain j for the following msgfem_local_spaces calls:
 * X0 (device, [n2_j][ld] FP32, first ncols columns used, ncols <= 8) on the
 * B2 rows; the remaining columns of the width-8 start block are drawn from
 * the counter-based generator as in a cold start.  X0 must stay valid until
 * it is replaced; X0 = NULL restores the cold start of subdomain j.  With a
 * start block the Rayleigh-Ritz test starts once the basis holds the wanted
 * pairs (instead of the wanted pairs plus one block). */
msgfem_status msgfem_set_start_block(msgfem_h h, int j, const float* X0, int ld, int ncols);

#ifdef __cplusplus
}
#endif
#endif
