// Internal layout of a PTROM online model, shared by ptrom.cu (online step)
// and ptrom_build.cu (offline training).
#pragma once

#include <vector>

#include "common.cuh"

namespace ptrom {

constexpr int kPT = 512;  // threads per instance
constexpr int kMaxM = 128, kMaxMr = 256, kMaxNs = 512, kMaxNc = 1 << 20;
constexpr int kTileB = 16;  // bodies per A C tile (32 dofs)

struct DevModel {
    int ns, M, Mr, Nc, Mp, Mrp;
    double dt, delta, tol;
    int max_gn, qr64;
    const float *phiB;  // [2ns][Mp]
    const float *x0B;   // [2ns]   relative to origin
    const float *phiT;  // [2Nc][Mp]
    const float *x0T;   // [2Nc]   relative to origin
    const float *gT;    // [Nc]    Gamma~ / (2 pi)
    const float *uB;    // [2ns]   dt times the superimposed inflow at the sampled dofs (zeros: none)
    const int *off, *idx;
    const float *At;    // [2ns][Mrp]  (A transposed, zero padded)
    int nlist;          // off[ns]: cluster-list entries
    int cache_rows;     // Phi_s and A^T staged in shared memory for the whole launch
    int cache_idx;      // the cluster lists staged in shared memory as 16-bit indices
    int xq_global;      // x^QT (and Gamma~) too large for shared memory: x^QT lives in the
                        // instance's state buffer after the state proper, Gamma~ is read from gT
};

struct InstArgs {
    DevModel m;
    double *state;  // [M] xhat, [2ns] carried velocity, [8] flags (as doubles)
    double *xhat;
    double *hist;
};

}  // namespace ptrom

struct ptrom_model {
    ptrom::DevModel d;
    int device;
    double ox, oy;
    std::vector<void *> bufs;
    size_t smem;
    // host FP64 copies of the description (kept for ptrom_save)
    int qr_prec = 0;
    std::vector<double> h_phi_s, h_x0_s, h_phi_c, h_x0_c, h_gamma_c, h_A;
    std::vector<double> h_u_s;  // [2 n_s] superimposed inflow at the sampled dofs (empty: none)
    std::vector<int> h_off, h_idx;
    // offline data, kept by models made with ptrom_build
    bool built = false;
    int n = 0;
    std::vector<double> phi;      // [2n][M] row-major
    std::vector<double> sigma;    // [M]
    std::vector<int> sampled;     // [n_s]
    std::vector<double> A;        // [M_r][2 n_s] row-major
    std::vector<int> cl_off;      // [N_c + 1] cluster -> members (CSR)
    std::vector<int> cl_mem;
    std::vector<double> x0_full;  // [2n] the current parameter's x^0 (host copy of x0_dev)
    std::vector<double> phi_r;    // [2n][M_r] row-major: the residual basis (Stage 3b)
    std::vector<double> tier2_traj;  // [n_params][steps + 1][M]: Tier-II reduced trajectories
    int n_params = 0, steps = 0;
    double *phi_dev = nullptr;    // [2n][M] FP64 (reconstruction)
    double *x0_dev = nullptr;     // [2n]
};

namespace ptrom {
// Bytes of an instance's state proper (xhat, carried velocity, flags), 256-byte
// aligned; a model with xq_global keeps 2 N_c floats of x^QT after it.
__host__ __device__ inline size_t state_base_bytes(int M, int ns) { return ((size_t)(M + 2 * ns + 8) * 8 + 255) & ~size_t(255); }
// Fill the parameter-dependent device arrays of a model from host arrays.
int model_fill_param(ptrom_model *m, const double *x0_s, const double *phi_c, const double *x0_c,
                     const double *gamma_c);
// Set the superimposed inflow at the sampled dofs (host [2 n_s]; nullptr
// clears it).
int model_fill_inflow(ptrom_model *m, const double *u_s);
// Give a built model its FP64 basis and reference state on the device
// (reconstruction); phi [2n][M] row-major, x0 [2n], host arrays.
int model_store_basis(ptrom_model *m, const double *phi, const double *x0);
}  // namespace ptrom
