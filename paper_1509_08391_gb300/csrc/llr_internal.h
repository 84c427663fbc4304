// llr_internal.h -- launch wrappers shared by the translation units of the
// CUDA library (not part of the public C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "llr_device.cuh"

namespace llr {

// Work programs of the persistent kernel.  Sweeps and RM create one work
// item per (composite sweep, lattice); every other program one item per
// lattice.
enum Program : int {
    kProgSweeps = 0,    // n_therm + n_meas composite sweeps at fixed a, optional measurement
    kProgRM = 1,        // the same, then the Robbins-Monro update of a
    kProgApproach = 2,  // approach sweeps until E lies in the window
    kProgResync = 3,    // fresh energy -> tracked energy
    kProgPass = 4,      // one heat-bath (pass_kind 0), overrelaxation (1) or multicanonical
                        // heat-bath (2) pass, no resync; or (3) the end of a composite sweep
    kProgBegin = 5,     // plain form: take a from a_in, clear the measurement
    kProgFinish = 6,    // plain form: resync + optional measurement + sweep counter
    kProgUpdate = 7,    // plain form: Robbins-Monro update from the accumulated measurement
    kProgMuca = 8,      // multicanonical composite sweeps (weight 1/rho~), energy history
};

struct KernelArgs {
    LatState *lats;
    float *theta;
    int n_lat;            // lattices in this launch (items per sweep)
    const int *order;     // nullable: slot i is lattice order[i]
    int program;
    int n_therm, n_meas, measure;
    int rm_index;
    const double *a_in;   // nullable: keep LatState::a
    double *a_out;        // RM / update: new a (nullable)
    double *mean_out;     // RM / update: <<dE>>; sweeps: sum of dE (nullable)
    int max_approach;
    double beta_up, beta_dn;
    int *approach_sweeps; // nullable
    int n_or;
    int block;            // window-accept block size B (power of two, <= 32)
    int pass_kind;        // pass: 0 heat-bath, 1 overrelaxation, 2 multicanonical, 3 end of sweep
    int class_mask;       // pass: bit c selects class c = 2 mu + parity
    // work queue (device): [0] error word (sticky across launches, cleared by
    // the host when it reads it), [1] item counter, [2 ..] sweeps done per slot
    unsigned *sync;
    unsigned long long wait_limit_ns;   // bounded wait for a lattice's previous sweep
    // graph replays: the Robbins-Monro step number lives in device memory
    const int *step_dev;  // nullable: rm_index += *step_dev, history row *step_dev
    double *hist;         // nullable: hist[step * n_lat + lattice] = new a
    // multicanonical weight 1/rho~ (pass kind 2 and kProgMuca): ln rho~ at the
    // edges e0 + k de (muca_n + 1 values) and the slope of each interval
    const double *muca_lnr;
    const double *muca_a;
    int muca_n;
    double muca_e0, muca_de, muca_a0;
    double *e_hist;       // kProgMuca, nullable: e_hist[sweep * n_lat + lattice] = E
    int ring;             // stages of the heat-bath ring in use (1, 2 or 4; set at launch)
};

// *step += 1 (the last node of a captured Robbins-Monro step).
cudaError_t launch_step_increment(int *step, cudaStream_t s);

struct LaunchCfg {
    int threads = 256;    // 128, 160, 192, 256 or 512: one consumer warp, the rest producers
    bool fast_math = true;
    int ring = 4;         // stages of the heat-bath producer/consumer ring in use: 1, 2 or 4
    int carveout = -1;    // shared-memory carve-out preference in percent, -1 = default
};

// Query (and cache) the resident-CTA count of a kernel variant; call before a
// stream capture so the capture itself makes no occupancy queries.
void prime_launch(const LaunchCfg &cfg);

// Reset the work queue and launch the persistent kernel (stream ordered);
// grid_out (nullable) receives the number of CTAs launched.
cudaError_t launch_llr(const KernelArgs &a, const LaunchCfg &cfg, cudaStream_t s,
                       int *grid_out = nullptr);

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

// One replica-exchange round over disjoint pairs of lattices (device arrays:
// pairs int[2 n_pairs], a double[n_lat], accepted int[n_pairs] or null).
cudaError_t launch_replica_exchange(LatState *lats, const int *pairs, int n_pairs,
                                    const double *a, uint32_t round, int *accepted,
                                    cudaStream_t s);

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

// Multicanonical reweighting kernels (Sec. 2.6, eq. (2.56)): ln rho~ of the
// table (lnr[n + 1] at the edges, slopes a[n]) at ns samples; moments of the
// samples reweighted to n_beta couplings (device beta[n_beta]; gx sample
// blocks per coupling, part = 4 gx n_beta doubles of scratch; outputs
// device double[n_beta] or null); tunnellings of n_chains chains.
cudaError_t launch_muca_lnrho(long long ns, const double *E, const double *lnr, const double *a,
                              int n, double e0, double de, double *out, int grid,
                              cudaStream_t s);
cudaError_t launch_reweight(long long ns, const double *E, const double *lr, double shift,
                            int n_beta, const double *beta, int gx, double *part, double *E1,
                            double *E2, double *var, cudaStream_t s);
cudaError_t launch_tunnellings(int n_steps, int n_chains, const double *E, double lo, double hi,
                               int *out, cudaStream_t s);

}  // namespace llr
