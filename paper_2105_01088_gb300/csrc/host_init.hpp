// Seeded initial states generated inside the library (host side, at admission):
// random pure covariances Gamma = O J O^T with O Haar-distributed on O(2N) and
// det O equal to the requested parity, and unit-modulus amplitudes.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC11), key = the 64-bit seed.  For state mu the
// n x n standard-normal matrix Z takes its entries 2j and 2j+1 (row-major) from
// counter (j, mu, 0, 0) by Box-Muller on the first two output words:
//   u1 = (x0 + 1) 2^-32, u2 = x1 2^-32, r = sqrt(-2 ln u1),
//   Z_2j = r cos(2 pi u2), Z_2j+1 = r sin(2 pi u2);
// the phase of lambda_mu is 2 pi x0 2^-32 from counter (0, mu, 1, 0).
// O = Q diag(sign R_ii) from the Householder QR of Z (the Haar measure), with its
// first column negated if det O differs from the parity.
#pragma once
#include <cmath>
#include <cstdint>
#include <thread>
#include <vector>

namespace sgs {

struct Philox4x32 {
    static void round(uint32_t x[4], uint32_t k0, uint32_t k1) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * x[0], p1 = (uint64_t)0xCD9E8D57u * x[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
        x[0] = y0; x[1] = lo1; x[2] = y2; x[3] = lo0;
    }
    // ten rounds, the key bumped by the Weyl constants between rounds
    static void block(uint32_t x[4], uint64_t key) {
        uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
        for (int r = 0; r < 10; r++) {
            if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
            round(x, k0, k1);
        }
    }
};

// state mu: Gamma (n x n, row-major) and lambda (re, im)
inline void seeded_state(int n, int mu, uint64_t seed, int parity, double* gamma, double* lambda) {
    const double two32 = 4294967296.0, twopi = 6.283185307179586476925286766559;
    std::vector<double> Z((size_t)n * n);
    for (size_t j = 0; j < (size_t)n * n / 2; j++) {
        uint32_t x[4] = {(uint32_t)j, (uint32_t)mu, 0u, 0u};
        Philox4x32::block(x, seed);
        const double u1 = ((double)x[0] + 1.0) / two32, u2 = (double)x[1] / two32;
        const double r = std::sqrt(-2.0 * std::log(u1));
        Z[2 * j] = r * std::cos(twopi * u2);
        Z[2 * j + 1] = r * std::sin(twopi * u2);
    }
    // Householder QR: column k's reflector v_k (stored below the diagonal of Z, scaled so
    // that v_k[k] = 1), R on and above the diagonal
    std::vector<double> beta(n, 0.0);
    int reflections = 0;
    for (int k = 0; k < n; k++) {
        double nrm = 0.0;
        for (int i = k; i < n; i++) nrm += Z[(size_t)i * n + k] * Z[(size_t)i * n + k];
        nrm = std::sqrt(nrm);
        const double akk = Z[(size_t)k * n + k];
        if (nrm == 0.0) continue;
        const double alpha = akk >= 0.0 ? -nrm : nrm;          // R_kk
        const double v0 = akk - alpha;
        for (int i = k + 1; i < n; i++) Z[(size_t)i * n + k] /= v0;
        beta[k] = -v0 / alpha;                                  // H = I - beta v v^T, v[k] = 1
        Z[(size_t)k * n + k] = alpha;
        reflections++;
        for (int j = k + 1; j < n; j++) {
            double s = Z[(size_t)k * n + j];
            for (int i = k + 1; i < n; i++) s += Z[(size_t)i * n + k] * Z[(size_t)i * n + j];
            s *= beta[k];
            Z[(size_t)k * n + j] -= s;
            for (int i = k + 1; i < n; i++) Z[(size_t)i * n + j] -= s * Z[(size_t)i * n + k];
        }
    }
    // Q = H_0 H_1 ... H_{n-1} applied to the identity (backward accumulation)
    std::vector<double> Q((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++) Q[(size_t)i * n + i] = 1.0;
    for (int k = n - 1; k >= 0; k--) {
        if (beta[k] == 0.0) continue;
        for (int j = k; j < n; j++) {
            double s = Q[(size_t)k * n + j];
            for (int i = k + 1; i < n; i++) s += Z[(size_t)i * n + k] * Q[(size_t)i * n + j];
            s *= beta[k];
            Q[(size_t)k * n + j] -= s;
            for (int i = k + 1; i < n; i++) Q[(size_t)i * n + j] -= s * Z[(size_t)i * n + k];
        }
    }
    // O = Q diag(sign R_ii); det O = (-1)^reflections prod sign R_ii
    int det = (reflections % 2) ? -1 : 1;
    for (int k = 0; k < n; k++) {
        if (Z[(size_t)k * n + k] < 0.0) {
            det = -det;
            for (int i = 0; i < n; i++) Q[(size_t)i * n + k] = -Q[(size_t)i * n + k];
        }
    }
    if (det != parity)
        for (int i = 0; i < n; i++) Q[(size_t)i * n] = -Q[(size_t)i * n];
    // Gamma = O J O^T, J = (+) [[0, 1], [-1, 0]]: Gamma_ij = sum_m (O_i,2m O_j,2m+1 - O_i,2m+1 O_j,2m)
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double s = 0.0;
            for (int m = 0; m < n / 2; m++)
                s += Q[(size_t)i * n + 2 * m] * Q[(size_t)j * n + 2 * m + 1] -
                     Q[(size_t)i * n + 2 * m + 1] * Q[(size_t)j * n + 2 * m];
            gamma[(size_t)i * n + j] = s;
        }
    uint32_t x[4] = {0u, (uint32_t)mu, 1u, 0u};
    Philox4x32::block(x, seed);
    const double th = twopi * (double)x[0] / two32;
    lambda[0] = std::cos(th);
    lambda[1] = std::sin(th);
}

// all M states, spread over the host's cores
inline void seeded_states(int n, int M, uint64_t seed, int parity, double* gamma, double* lambda) {
    const int nt = std::max(1, std::min<int>(M, (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; t++)
        pool.emplace_back([=] {
            for (int mu = t; mu < M; mu += nt)
                seeded_state(n, mu, seed, parity, gamma + (size_t)mu * n * n, lambda + 2 * mu);
        });
    for (auto& th : pool) th.join();
}

}  // namespace sgs
