// Definitions shared by the single-image and the batched 2D TV-l2 drivers.
#pragma once
#include <math.h>

namespace tvk {

// Step sizes of eq. pd at iteration k (accelerated variant, gamma = 1,
// tau_0 = sigma_0 = 1): tau_k, sigma_k, theta_{k-1}, tau_{k-1}.
struct Tv2dParams {
    double tau, sigma, theta_prev, tau_prev;  // tau_k, sigma_k, theta_{k-1}, tau_{k-1}
};

// They are computed on the host in FP64 and passed to the device by value, 256
// per launch.
constexpr int kParamChunk = 256;
struct ParamChunk {
    int first, count;
    Tv2dParams p[kParamChunk];
};


// Host: fill `chunk` with entries first .. first+count-1 of the schedule.
inline void fill_params(ParamChunk &chunk, int first, int count)
{
    double tau = 1.0, sigma = 1.0, theta_prev = 0.0, tau_prev = 1.0;
    for (int k = 0; k < first + count; ++k) {
        if (k >= first) chunk.p[k - first] = Tv2dParams{tau, sigma, theta_prev, tau_prev};
        const double theta = 1.0 / sqrt(1.0 + 2.0 * tau);
        tau_prev = tau;
        tau *= theta;
        sigma /= theta;
        theta_prev = theta;
    }
    chunk.first = first;
    chunk.count = count;
}

}  // namespace tvk
