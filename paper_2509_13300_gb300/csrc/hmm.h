// Profile-HMM scoring by the warp wavefront (hmm.cu): the launch, its device
// scratch and the choice between it and the block-per-group kernel that
// launch_hmm_score (ah_internal.h) starts.
#pragma once

#include "ah_internal.h"

namespace ah {

// True when a score (Forward if `forward`, else Viterbi) runs on the warp
// wavefront: by default the Forward scores; AH_HMM_KERNEL=wave or =rows forces
// one kernel for both scores (a profiling aid).
bool hmm_use_wave(bool forward);

// Device scratch of launch_hmm_wave in bytes: one stripe-boundary buffer of
// 3 * (max_len + 1) floats per warp of its grid (at most 256 MB beyond one
// block per SM).
size_t hmm_scratch_bytes(uint64_t n, int max_len, int sms);

// The scores of n amplicons, as launch_hmm_score computes them, by the warp
// wavefront; bnd holds hmm_scratch_bytes(n, max_len, sms) bytes.
void launch_hmm_wave(const ah_amplicon *amps, const uint32_t *order, uint64_t n, const uint32_t *planes,
                     const uint64_t *contig_off, uint32_t n_contigs, const float *t, const float *e, int m,
                     int max_len, bool forward, float *bnd, float *score_out, int *err, int sms, cudaStream_t s);

} // namespace ah
