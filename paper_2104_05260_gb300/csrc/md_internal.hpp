// State and launch interface of the MD loop (md.cu, md.cpp).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hsma {

enum { MD_FLAG_CELL_OVERFLOW = 1, MD_FLAG_LEFT_SLAB = 2 };
constexpr int MD_THERMO_COLS = 6;   // K, U_LJ, U_coulomb, xi, eta, extended energy

// Device-resident scalars of a run.
struct MdScalars {
  double xi, eta;          // thermostat variable and its time integral
  double vscale;           // pending velocity scale (thermostat halves) for the next kick
  double vscale_end;       // scale that makes the stored velocities this step's
  double last_K, last_U;
  long long step;          // thermo rows written in this run
  long long rdf_samples;
  int flags;
};

struct MdArgs {
  int N;
  double L[3];
  double* x;            // N*3, wrapped into [0, L)
  double* v;            // N*3 (before vscale_end)
  int* img;             // N*3 image counters
  const double* q;      // N
  double* f_lj;         // N*3
  const double* f_c;    // N*3, Coulomb forces (electrostatics' output)
  const double* coul_energy;   // device scalar (electrostatics' energy) or null
  double* blk_k;        // per-block sums of v^2
  double* blk_u;        // per-block LJ energy (md_lj_blocks entries)
  MdScalars* sc;
  double* thermo;       // thermo_cap rows of MD_THERMO_COLS
  long long thermo_cap;
  // cell list
  int nc[3];
  double inv_w[3];      // cells per unit length
  int cap;              // particles per cell
  int* cell_count;
  int* cell_list;
  // parameters
  double dt, half_dt_m, mass;
  double sigma2, eps, rc2;
  int thermostat;
  double g_kT, Q;
  // RDF
  unsigned long long* rdf;   // 3 * rdf_bins
  int rdf_bins;
  double rdf_rmax;
  // slab (Sec. 4.3): periodic in x, y; LJ walls at z = 0 and z = L[2]
  int slab;
  double wall_sigma, wall_eps, wall_rc;
  unsigned long long* zhist;  // 2 * zhist_bins: cations, anions over (0, L[2])
  int zhist_bins;
};

int md_blocks(int N);      // blocks of the per-particle kernels (blk_k entries)
int md_lj_blocks(int N);   // blocks of the LJ kernel (blk_u entries)
cudaError_t md_launch_kick_drift(const MdArgs& a, cudaStream_t s);
cudaError_t md_launch_lj(const MdArgs& a, int n_cells, cudaStream_t s);
cudaError_t md_launch_kick_finish(const MdArgs& a, cudaStream_t s);
cudaError_t md_launch_start(const MdArgs& a, cudaStream_t s);
cudaError_t md_launch_rdf(const MdArgs& a, cudaStream_t s);

}  // namespace hsma
