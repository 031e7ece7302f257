// Launchers of the noise-reduction kernels (Section V).
#pragma once

#include <cuda_runtime.h>

namespace ds {

// halo (voxels per side) the Lanczos stencil needs: ceil(m m'/2) - 1
int lanczos_halo(int m, int mprime);

// ext: I(G) on the grid extended by the halo on every side, [cnt+2h]^3 (C order);
// tmp1, tmp2: scratch of the same size; out: [cnt0][cnt1][cnt2]
template <typename T>
void lanczos_resample(const T *ext, T *tmp1, T *tmp2, T *out, const int cnt[3], int m, int mprime, cudaStream_t s);

// ext as above, w: normalised (2h+1)^3 stencil on the device; out: [cnt0][cnt1][cnt2]
template <typename T>
void sphere_resample(const T *ext, const T *w, T *out, const int cnt[3], int h, cudaStream_t s);

}  // namespace ds
