// The learned warm start's choice of initial iterates.  Per load case the
// solve starts from whichever candidate has the smallest true residual
// ||f_i - K x_i||: zero, the previous design iteration's solution, the
// predictor's scale * y_i, or the previous solution plus the change of the
// prediction since the previous iteration.  Candidates are shifted to zero
// mean (the periodic operator's null space is the constants).
#pragma once
#include "kernels_fine.cuh"

namespace otm {

enum { kWsZero = 0, kWsPrev = 1, kWsNet = 2, kWsDelta = 3 };

struct WsState {
    double cand[4][6];   // per candidate: ||f_i - K x_i||^2 (i < 3), ||f_i||^2
    double best[3];
    int choice[3];
    int pad;
};

struct FinStore {
    double* out;
    __device__ void operator()(const double* s) const {
        for (int i = 0; i < 6; ++i) out[i] = s[i];
    }
};

// xc = scale * y (NET) or x + xl + scale * (y - y_prev) (DELTA)
template <class R>
__global__ void __launch_bounds__(256)
k_ws_cand(size_t N, int mode, const R* __restrict__ x, const R* __restrict__ xl, const float* __restrict__ y,
          const float* __restrict__ yp, double scale, R* __restrict__ xc) {
    using C = typename St<R>::C;
    const C sc = (C)scale;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * N; e += (size_t)gridDim.x * blockDim.x) {
        if (mode == kWsNet) {
            xc[e] = sc * (C)y[e];
        } else {
            C b = x[e];
            if (xl) b += xl[e];
            xc[e] = b + sc * ((C)y[e] - (C)yp[e]);
        }
    }
}

// Per load case, the candidate with the smallest residual (ties keep the
// earlier of zero, previous, change, predictor).
static __global__ void k_ws_decide(WsState* ws, int have_prev, int have_delta) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i < 3; ++i) {
        double best = ws->cand[kWsNet][3 + i];   // zero start: residual f
        int ch = kWsZero;
        if (have_prev && ws->cand[kWsPrev][i] < best) {
            best = ws->cand[kWsPrev][i];
            ch = kWsPrev;
        }
        if (have_delta && ws->cand[kWsDelta][i] < best) {
            best = ws->cand[kWsDelta][i];
            ch = kWsDelta;
        }
        if (ws->cand[kWsNet][i] < best) {
            best = ws->cand[kWsNet][i];
            ch = kWsNet;
        }
        ws->best[i] = best;
        ws->choice[i] = ch;
    }
}

// Install the chosen starts into the solution pair (x, xl).
template <class R>
__global__ void __launch_bounds__(256)
k_ws_take(size_t N, const WsState* __restrict__ ws, const R* __restrict__ xnet, const R* __restrict__ xdelta,
          R* __restrict__ x, R* __restrict__ xl) {
    const int c0 = ws->choice[0], c1 = ws->choice[1], c2 = ws->choice[2];
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * N; e += (size_t)gridDim.x * blockDim.x) {
        const int i = e < N ? 0 : (e < 2 * N ? 1 : 2);
        const int ch = i == 0 ? c0 : (i == 1 ? c1 : c2);
        if (ch == kWsPrev) continue;
        x[e] = ch == kWsZero ? R(0) : (ch == kWsNet ? xnet[e] : xdelta[e]);
        if (xl) xl[e] = R(0);
    }
}

}  // namespace otm
