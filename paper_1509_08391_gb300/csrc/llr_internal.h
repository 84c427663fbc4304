// llr_internal.h -- launch wrappers shared by the translation units of the
// CUDA library (not part of the public C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "llr_device.cuh"

namespace llr {

enum ChainMode : int {
    kModeSweeps = 0,    // n_therm + n_meas sweeps at fixed a, optional measurement
    kModeRM = 1,        // the same, then the Robbins-Monro update of a
    kModeApproach = 2,  // approach sweeps until E lies in the window
    kModeResync = 3,    // fresh energy -> tracked energy, nothing else
    kModePass = 4,      // one heat-bath (pass_kind 0) or overrelaxation (1) pass, no resync
};

struct ChainArgs {
    LatState *lats;
    float *theta;
    int n_lat;
    int mode;
    int n_therm, n_meas, measure;
    int rm_index;
    const double *a_in;   // nullable: use LatState::a
    double *a_out;        // mode RM: new a;     nullable
    double *mean_out;     // mode RM: <<dE>>; mode sweeps: sum of dE; nullable
    int max_approach;
    double beta_up, beta_dn;
    int *approach_sweeps; // nullable
    int n_or;
    int block;            // window-accept block size B (power of two, <= 32)
    const int *order;     // nullable: CTA i works on lattice order[i]
    int pass_kind;        // mode pass: 0 heat-bath, 1 overrelaxation
    int class_mask;       // mode pass: bit c selects class c = 2 mu + parity
};

// Batched launch: one CTA per lattice, whole work of `mode` in one kernel.
cudaError_t launch_chain(const ChainArgs &a, int threads, bool fast_math, cudaStream_t s);

// Plain form: single-lattice kernels, one launch per pass / resync / update.
cudaError_t launch_plain_pass(const ChainArgs &a, int lattice, int kind, double a_val,
                              cudaStream_t s);
cudaError_t launch_plain_finish(const ChainArgs &a, int lattice, int measure_this,
                                cudaStream_t s);
cudaError_t launch_plain_update(const ChainArgs &a, int lattice, cudaStream_t s);
cudaError_t launch_plain_begin(const ChainArgs &a, int lattice, cudaStream_t s);

// Hot start of every link of every lattice.
cudaError_t launch_hot_start(LatState *lats, float *theta, int n_lat, int max_half,
                             cudaStream_t s);

// Set the tracked energy of one lattice from an FP64 energy (device scalar).
cudaError_t launch_set_energy(LatState *lat_dev, const double *E_dev, cudaStream_t s);

// FP64 fresh energies.
cudaError_t launch_energy_fp64(const LatState *lats, const float *theta, int n_lat,
                               double *E_out, cudaStream_t s);

// Canonical (mu*V + s) <-> internal layout of one lattice.
cudaError_t launch_to_canonical(const LatState *lat_dev, const float *theta, float *out,
                                int n_links, cudaStream_t s);
cudaError_t launch_from_canonical(const LatState *lat_dev, float *theta, const float *in,
                                  int n_links, cudaStream_t s);

// Record the message returned by llr_last_error() on this thread; returns code.
int set_last_error(int code, const char *msg);

// Reconstruction kernels.
cudaError_t launch_lnrho(int n, const double *c, const double *a, double *out, cudaStream_t s);
cudaError_t launch_observables(int n, const double *c, const double *a, int n_beta,
                               const double *beta, double *lnZ, double *E1, double *E2,
                               cudaStream_t s);
cudaError_t launch_cv_peak(int n, const double *c, const double *a, double beta_lo,
                           double beta_hi, int n_grid, double tol, double *out,
                           cudaStream_t s);

}  // namespace llr
