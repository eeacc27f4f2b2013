/*
 * fkreg_sweep.h - bandwidth sweeps with a Fourier period per group.
 *
 * A plan represents every bandwidth of its list with one Fourier period,
 * P_j >= (hi_j - lo_j) + the kernel tail of the WIDEST bandwidth (so no
 * periodic image reaches the box), and one type-1 spectrum whose modes reach
 * the spectral extent of the NARROWEST bandwidth (Sec. 1.2, eqs. 16-21).
 * The number of modes grows with P / sigma, so on a sweep such as sixteen
 * bandwidths log-spaced over a decade the narrow bandwidths pay for the wide
 * bandwidths' period: their type-1 and type-2 grids are larger than their
 * own tail requires (for the 3-D sweep of sigma 0.01 .. 0.1 on the unit
 * cube, 588^3 fine cells at P = 1.587 where P = 1.19 needs 448^3).
 *
 * A sweep splits the bandwidth list into contiguous groups, one plan per
 * group, each with the period and spectra its own bandwidths need, and runs
 * the groups one after another on the caller's stream.  The groups share
 * nothing but the inputs: each sorts the samples for its own fine grid
 * (about half a millisecond for 4e6 samples), spreads them and transforms
 * its spectra.  Probes drawn on the device are functions of the seed, the
 * probe index and the ORIGINAL sample index, so every group smooths the
 * same probe vectors.  The split minimises a cost model of the step (per
 * group: spreading N w^d strengths, transforming the type-1 grid; per
 * bandwidth: the type-2 grid, its transform and gather) calibrated on GB300
 * measurements; a split is taken only when it cuts the modelled cost.  A
 * Gaussian group whose bandwidths hold few samples within the cut radius is
 * given direct sums (FKREG_KERNEL_GAUSSIAN_DIRECT) when the model finds them
 * cheaper than its NUFFT; a sweep over a compact kernel is one group.
 *
 * Outputs have the layouts of fkreg_smooth / fkreg_df / fkreg_variance
 * (leading dimension n_bw, the caller's bandwidth order): each group writes
 * its bandwidths' slices.  Entry points mirror the plan's; what a group plan
 * returns is returned, with the message of the group that failed in
 * fkreg_sweep_last_error.
 */
#ifndef FKREG_SWEEP_H
#define FKREG_SWEEP_H

#include <stddef.h>
#include <stdint.h>

#include "fkreg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fkreg_sweep_s* fkreg_sweep;

/*
 * Create a sweep for up to max_n samples.  opts as for fkreg_plan_create
 * (Gaussian regression kernel only: the compact kernels have no Fourier
 * period).  max_groups >= 1 bounds the number of groups (1 gives one plan,
 * the same as fkreg_plan_create); groups are contiguous index ranges of
 * opts->H.  Needs a current CUDA device; allocates no device memory.
 * Returns FKREG_ERR_INVALID_ARG / FKREG_ERR_UNSUPPORTED as plan creation
 * does (message in fkreg_global_error()).
 */
fkreg_status fkreg_sweep_create(const fkreg_opts* opts, int64_t max_n, int max_groups,
                                fkreg_sweep* out);

/*
 * Host-only (no CUDA call): the split fkreg_sweep_create chooses for these
 * arguments.  *n_groups groups; first_bw (array of n_bw + 1, may be NULL)
 * receives the first bandwidth of each group and then n_bw; group_kernel
 * (array of n_bw, may be NULL) the regression kernel of each group's plan
 * (for a Gaussian sweep FKREG_KERNEL_GAUSSIAN, the NUFFT, or
 * FKREG_KERNEL_GAUSSIAN_DIRECT, direct sums, whichever the cost model finds
 * cheaper for the group); *modelled_s (may be NULL) the model's seconds.
 */
fkreg_status fkreg_sweep_split(const fkreg_opts* opts, int64_t max_n, int max_groups,
                               int* n_groups, int* first_bw, int* group_kernel,
                               double* modelled_s);

/*
 * The split: *n_groups groups; first_bw[g] (array of n_groups + 1, may be
 * NULL) is the first bandwidth of group g, first_bw[n_groups] = n_bw;
 * group_kernel[g] (may be NULL) its plan's regression kernel; geoms[g]
 * (array of n_groups, may be NULL) the group plan's geometry.  Call once
 * with the arrays NULL to learn n_groups.
 */
fkreg_status fkreg_sweep_groups(fkreg_sweep S, int* n_groups, int* first_bw, int* group_kernel,
                                fkreg_geometry* geoms);

/* Device bytes of the sweep's workspace (the groups' workspaces, each 256-byte aligned). */
fkreg_status fkreg_sweep_workspace_bytes(fkreg_sweep S, size_t* bytes);

/* Hand the sweep its workspace (device, 256-byte aligned, caller-owned); as
 * fkreg_set_workspace for every group. */
fkreg_status fkreg_sweep_set_workspace(fkreg_sweep S, void* ws, size_t bytes, void* stream);

/* fkreg_set_points for every group (each sorts for its own fine grid). */
fkreg_status fkreg_sweep_set_points(fkreg_sweep S, int64_t n, const void* x_dev, void* stream);

/* fkreg_smooth / fkreg_df over every group; `out` as for the plan calls,
 * for all n_bw bandwidths. */
fkreg_status fkreg_sweep_smooth(fkreg_sweep S, const void* y_dev, const fkreg_outputs* out,
                                void* stream);
fkreg_status fkreg_sweep_df(fkreg_sweep S, const void* y_dev, int n_probes, uint64_t seed,
                            const void* probes_dev, const fkreg_outputs* out, void* stream);

/* fkreg_variance over every group: mhat_at_x_dev [n_bw][n_rhs][n] from the
 * last fkreg_sweep_smooth / fkreg_sweep_df, sigma2_grid_dev [n_bw][n_rhs][M]. */
fkreg_status fkreg_sweep_variance(fkreg_sweep S, const void* y_dev, const void* mhat_at_x_dev,
                                  void* sigma2_grid_dev, void* stream);

/* fkreg_log_variance over every group (eqs. 24-26); arrays as for the plan
 * call, for all n_bw bandwidths. */
fkreg_status fkreg_sweep_log_variance(fkreg_sweep S, const void* y_dev, const void* mhat_at_x_dev,
                                      void* v_grid_dev, void* v_at_x_dev, double* kappa_dev,
                                      void* sigma2_grid_dev, void* stream);

/* fkreg_backward for bandwidth b (index in the caller's list): GCV of
 * eq. 22 with the Monte-Carlo trace of Sec. 2.1 and its gradient with
 * respect to log h, y and x, run by the plan of b's group (whose opts carry
 * FKREG_WANT_BACKWARD if the sweep's did); arguments, outputs and the
 * plan-level refusals as for fkreg_backward; b outside [0, n_bw) returns
 * FKREG_ERR_INVALID_ARG before anything runs. */
fkreg_status fkreg_sweep_backward(fkreg_sweep S, const void* y_dev, int n_probes, uint64_t seed,
                                  const void* probes_dev, int b, double* gcv_dev,
                                  double* dlogh_dev, void* dy_dev, void* dx_dev, void* stream);

/* fkreg_sync_status of every group (the first failure is returned). */
fkreg_status fkreg_sweep_sync_status(fkreg_sweep S, void* stream);

/* fkreg_set_timing for every group; fkreg_stage_times summed over the groups
 * (arrays as for fkreg_stage_times). */
fkreg_status fkreg_sweep_set_timing(fkreg_sweep S, int enable);
fkreg_status fkreg_sweep_stage_times(fkreg_sweep S, double* ms, int64_t* launches,
                                     int64_t* kernel_launches);

const char* fkreg_sweep_last_error(fkreg_sweep S);
void fkreg_sweep_destroy(fkreg_sweep S);

#ifdef __cplusplus
}
#endif

#endif /* FKREG_SWEEP_H */
