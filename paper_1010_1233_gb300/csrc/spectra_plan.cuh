// Plan of one standalone correlator-sampling call (spectra_api.cu): a one-replica
// descriptor and the layout of the call's scratch memory.
#pragma once
#include "flb_internal.cuh"

namespace flb {

struct SpectraPlan {
  ReplicaDesc desc;
  int64_t n_vb_rows, n_vb_cols, n_vb_cols_a;
  int ncol, rows_block, rows_smem, cols_smem;
  int64_t off_desc, off_vb, off_tw_x, off_tw_y, off_spec;   // byte offsets in the scratch
  size_t scratch_bytes;
  int64_t n_sum_doubles;                                    // length of the pair-sum output
};

// Validate sizes and lay out the scratch (no device work).
int spectra_plan(int precision, int nx, int ny, int n_fields, SpectraPlan& plan);
// Store the plan into the scratch and launch the transforms and the accumulation.
int spectra_launch(int precision, SpectraPlan& plan, char* scratch, const void* fields, double* pair_sums,
                   double* mean0, cudaStream_t st);

}  // namespace flb
