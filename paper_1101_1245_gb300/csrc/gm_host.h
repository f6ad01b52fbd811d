// Host-side declarations shared by the gpumcd library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gm_common.cuh"

namespace gm {

// Energy bounds of the two table grids (MeV).
struct TableGeom {
    double p0, p1;  // photon grid
    double e0, e1;  // electron grid
};

Grid make_grid(const TableGeom &g);

cudaError_t launch_build_tables(const gpumcd_material *mats, int n_mat, const TableGeom &g,
                                double t_c, double k_c, float *d_tab, cudaStream_t s);
cudaError_t launch_grid_energies(const TableGeom &g, float *out, cudaStream_t s);
cudaError_t launch_pack_phantom(const uint8_t *mat, const float *rho, uint64_t nvox, int n_mat,
                                uint32_t *vox, unsigned int *rho_max_bits, int *bad, cudaStream_t s);
cudaError_t launch_majorants(const float *tab, const unsigned int *rho_max_bits, int n_mat, float *maj,
                             cudaStream_t s);
cudaError_t launch_spectrum(const double *edges, const double *w, int n, float *out, cudaStream_t s);
cudaError_t launch_fold(const unsigned long long *tally, const uint32_t *vox, uint64_t nvox, int W,
                        const double *n_b, double n_tot, double inv_vol, double *dose, double *sigma,
                        unsigned long long *dmax_bits, unsigned long long *dep_sum, int n_sm, cudaStream_t s);
// Blocks of the s_thr reduction for nvox voxels: its partials take 16 bytes each.
int sthr_blocks(uint64_t nvox, int n_sm);
cudaError_t launch_sthr(const double *dose, const double *sigma, uint64_t nvox,
                        const unsigned long long *dmax_bits, double thr, double *sum,
                        unsigned long long *count, void *part, int n_sm, cudaStream_t s);
cudaError_t launch_sum_u64(const unsigned long long *a, uint64_t n, unsigned long long *out, int n_sm,
                           cudaStream_t s);
cudaError_t launch_fold_noalloc(int device, const unsigned long long *tally, const uint32_t *vox, uint64_t nvox,
                                int W, const double *n_b, double n_tot, double inv_vol, double thr, double *dose,
                                double *sigma, cudaStream_t s, unsigned long long result[4]);
cudaError_t launch_philox(const uint32_t *ctr, uint2 key, uint64_t n, int curand, uint32_t *out,
                          cudaStream_t s);

// Transport (gm_transport.cu).
size_t transport_smem_bytes(uint32_t tab_bytes);
cudaError_t transport_configure();
cudaError_t launch_transport(const TransportArgs &a, int grid, int block, int blocks_per_sm, cudaStream_t s);
// The transport kernel launch_transport runs for these arguments and shape
// (null when no compiled kernel covers them).
const void *transport_kernel(const TransportArgs &a, int block, int blocks_per_sm);
// Claim order of a spectrum or phase space grouped by energy: order[0..n) =
// offsets j of the histories hist_base + j of plan P, in decreasing order of
// their primary's energy bin; count (GPUMCD_MAX_SPECTRUM_BINS unsigned) and
// keys (n uint16_t) are scratch.
cudaError_t launch_group_order(const PlanDev &P, uint32_t n, unsigned *count, uint16_t *keys, uint32_t *order,
                               cudaStream_t s);
cudaError_t launch_debug_sample(const float *tab, const Phys &phys, int kind, float p0, int material,
                                const float *spec, int n_spec, uint64_t n, uint64_t seed, float *out,
                                cudaStream_t s);

}  // namespace gm
