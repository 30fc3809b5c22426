// flb_obs.cuh -- argument blocks and launchers of the observable kernels.
#pragma once
#include "flb_internal.cuh"

namespace flb {

constexpr int NRED = 9;  // sum dev, sum j (3), sum psi, sum u^2 (3), non-finite count

struct DftArgs {
    const float *in;       // real input field
    long long off, sy, sz; // element offset of (0,0,0) and strides of y and z (x stride 1)
    int nx, ny, nz;        // extents
    int Kx, Ky, Kz;        // number of kept wavevector indices per axis
    float2 *X1, *X2;       // scratch: nz*ny*Kx and nz*Ky*Kx complex values
    double *S;             // accumulator Kz*Ky*Kx (may be null: no accumulation)
    double scale;          // factor on |.|^2
    float2 *snap = nullptr;  // if not null: the Fourier components, Kz*Ky*Kx
};

cudaError_t launch_totals(const Geom &g, int q, int storage, const void *f, const float *psi, const float *u,
                          double *partial, int nblocks, double *out, cudaStream_t s);
cudaError_t launch_dft_accumulate(const DftArgs &a, cudaStream_t s);
cudaError_t launch_heights(const Geom &g, const float *psi, float *h, cudaStream_t s);
// acc[l*K + k] += scale Re(ring[slot][k] conj(ring[slot - l][k])) for l < nlag (ring of L slots of K values)
cudaError_t launch_dyn_corr(const float2 *ring, int L, int slot, int nlag, long long K, double *acc, double scale,
                            cudaStream_t s);

}  // namespace flb
