// teuk_aux.cuh -- launchers of the post-processing kernels of teuk_aux.cu that work
// across instances (the others are declared in teuk_internal.cuh).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace teuk {

// One mode of a mode sum: its waveform ring ([cap][nth] records, time level t in slot
// t % cap) and its azimuthal number.
struct ModeRing {
    const double2* wave;
    int64_t cap;
    int m;
    int pad;
};

// Field of Eqs. (3)-(4) at the extraction radius, summed over modes:
//   out[k][j][l] = r3 sum_i e^{i m_i (phi[l] + shift)} W_i[first + k][j]
// with the modes added in index order (modes, phi, out: device arrays).
void launch_mode_sum(cudaStream_t st, const ModeRing* modes, int n_modes, int nth,
                     const double* phi, int n_phi, int64_t first, int64_t n_rec, double r3,
                     double shift, double2* out);

// Radiated fluxes of several modes (teuk_flux.cu): the modes' rings, the time step,
// the Boyer-Lindquist extraction radius r, the spin a and the phi~ shift of Eq. (3) at
// r; the records first .. first + R - 1 in chunks of Lc records (n_chunks of them, at
// most 65535); the rows in groups of RB (n_rg groups), K RB <= 256.
struct FluxDev {
    const ModeRing* modes;
    int K, nth;
    int64_t first, R;
    int Lc, n_chunks;
    int RB, n_rg;
    double dt, r, a, shift;
};
// Weights of one (mode, row) entry of the flux sums: w |F|^2, w cos(theta) |F|^2 and
// m w |F|^2 (w = sin(theta) dtheta, F the entry's factor).
struct alignas(32) FluxWeights {
    double e, z, jz, pad;
};
// Device buffers of one call: chunk totals and starts [n_chunks][K nth], the entries'
// weights g [K nth] and gp [K nth] (w sin(theta) F conj(F') with the partner's F'), the partner of each mode (the
// index of mode m+1, or -1) [K], the row groups' sums [R][n_rg][5] and the output
// [R][10].  Returns the number of kernels launched.
struct FluxScratch {
    double2 *totN, *totH, *stN, *stH;
    FluxWeights* g;
    double2* gp;
    const int* partner;
    double* part;
    double* out;
};
int launch_radiated_flux(cudaStream_t st, const FluxDev& f, const FluxScratch& s);

struct InstDev;
// Checked builds: submit the index one past the end of d's state plane to the bounds
// check (no access), setting the status word's bounds bit.
void launch_check_selftest(cudaStream_t st, const InstDev& d);

}  // namespace teuk
