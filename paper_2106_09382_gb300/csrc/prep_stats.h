// Column statistics of the data preparation over many CTAs (prep_gram.cu).
// Internal: not part of the C ABI.
#pragma once
#include "kernels.h"

namespace concord {

// As launch_col_stats, spread over many CTAs (row chunks summed per column,
// then combined in chunk order: deterministic); scratch holds
// col_stats_chunks(n) x p doubles.
int col_stats_chunks(int n);
cudaError_t launch_col_stats_chunked(const void* X, int x_f32, int n, int p, int ldx, int prep,
                                     double* mean, double* inv_scale, int* bad, double* scratch,
                                     cudaStream_t st);

}  // namespace concord
