// flb_obs.cuh -- argument blocks and launchers of the observable kernels.
#pragma once
#include "flb_internal.cuh"

namespace flb {

constexpr int NRED = 9;  // sum dev, sum j (3), sum psi, sum u^2 (3), non-finite count
constexpr int NMSQ = 20; // per-mode sums of m_k^2 (q <= 19) and a non-finite count

// Moment basis of one lattice in plane order, E[k*q + i] (Gram-Schmidt, built on the host).
struct ModeBasis {
    float E[19 * 19];
    int q;
};

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
// out[k] = sum over sites of m_k^2 (k < q), out[NMSQ-1] = non-finite count; partial holds nblocks*NMSQ
cudaError_t launch_mode_msq(const Geom &g, int storage, const ModeBasis &B, const void *f, double *partial,
                            int nblocks, double *out, cudaStream_t s);
cudaError_t launch_heights(const Geom &g, const float *psi, float *h, cudaStream_t s);
// acc[l*K + k] += scale Re(ring[slot][k] conj(ring[slot - l][k])) for l < nlag (ring of L slots of K values)
cudaError_t launch_dyn_corr(const float2 *ring, int L, int slot, int nlag, long long K, double *acc, double scale,
                            cudaStream_t s);

}  // namespace flb
