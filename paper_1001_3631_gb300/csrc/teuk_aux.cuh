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

struct InstDev;
// Checked builds: submit the index one past the end of d's state plane to the bounds
// check (no access), setting the status word's bounds bit.
void launch_check_selftest(cudaStream_t st, const InstDev& d);

}  // namespace teuk
