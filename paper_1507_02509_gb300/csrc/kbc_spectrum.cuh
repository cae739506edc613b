// Shell binning of the energy spectrum (kbc_spectrum in include/kbc.h).
#pragma once

#include <cuda_runtime.h>

namespace kbc {

// Adds the energy of one velocity component's half spectrum (cuFFT D2Z
// layout [n][n/2 + 1]: row = y wavenumber in FFT order, column = x
// wavenumber 0 .. n/2) to the shell sums E[round(|k|)], shells >= nbins left
// out.  scale = 1 / n^4 turns |FFT|^2 into |u_hat|^2 for coefficients
// normalised by the node count; a column 0 < kx < n/2 also stands for its
// Hermitian partner -kx (weight 2 x 1/2), columns 0 and n/2 for themselves
// (weight 1/2).  With smem != 0 each block first sums into a shared
// histogram of nbins doubles.
__global__ void spectrum_bin(const double2* __restrict__ uh, int n, int nbins, double scale,
                             double* __restrict__ E, int smem)
{
    extern __shared__ double hist[];
    if (smem) {
        for (int b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0.0;
        __syncthreads();
    }
    const int w = n / 2 + 1;
    const long long total = (long long)n * w;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int ky = (int)(q / w), kx = (int)(q - (long long)ky * w);
        const int fy = (2 * ky < n) ? ky : ky - n;
        const int shell = (int)rint(sqrt((double)kx * kx + (double)fy * fy));
        if (shell >= nbins) continue;
        const double2 c = uh[q];
        const double v = ((kx == 0 || 2 * kx == n) ? 0.5 : 1.0) * scale * (c.x * c.x + c.y * c.y);
        if (smem) atomicAdd(&hist[shell], v);
        else atomicAdd(&E[shell], v);
    }
    if (smem) {
        __syncthreads();
        for (int b = threadIdx.x; b < nbins; b += blockDim.x)
            if (hist[b] != 0.0) atomicAdd(&E[b], hist[b]);
    }
}

// Z(k) = (2 pi k / n)^2 E(k): the enstrophy density of shell k.
__global__ void spectrum_enstrophy(const double* __restrict__ E, double* __restrict__ Z, int nbins,
                                   int n)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
        const double k = 6.283185307179586 * (double)b / (double)n;
        Z[b] = k * k * E[b];
    }
}

}  // namespace kbc
