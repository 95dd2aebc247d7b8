// mv_icp.cuh -- the Gauss-Newton step of the point-to-plane ICP (FP64), for
// the host and the device: the 6x6 solve and the pose update by the twist.
#pragma once

#include <math.h>

namespace mv {

// T <- exp(x^) T for the twist x = (rho, phi): rotation by Rodrigues,
// translation V rho.  The coefficients sin(th)/th, (1 - cos th)/th^2 and
// (th - sin th)/th^3 come from their Maclaurin series in th^2 for th < 1e-2
// (the first omitted term is below 1e-27 relative: exact in double; the
// Gauss-Newton increments of tracking are that small), else from sin and cos.
// On the device this avoids the long serial FP64 sequences of sin, cos and
// sqrt on a pipe that B300 runs at a small fraction of its FP32 rate.
__host__ __device__ inline void apply_twist(const double x[6], double T[16])
{
    const double p0 = x[3], p1 = x[4], p2 = x[5];
    const double th2 = p0 * p0 + p1 * p1 + p2 * p2;
    double A, B, Cc;
    if (th2 < 1e-4) {
        // nested: the ratio of consecutive terms is th^2 / ((2k)(2k+1)) or / ((2k+1)(2k+2))
        const double q = th2;
        A = 1.0 - q * (1.0 / 6) * (1.0 - q * (1.0 / 20) * (1.0 - q * (1.0 / 42) * (1.0 - q * (1.0 / 72))));
        B = 0.5 * (1.0 - q * (1.0 / 12) * (1.0 - q * (1.0 / 30) * (1.0 - q * (1.0 / 56) * (1.0 - q * (1.0 / 90)))));
        Cc = (1.0 / 6) * (1.0 - q * (1.0 / 20) * (1.0 - q * (1.0 / 42) * (1.0 - q * (1.0 / 72) * (1.0 - q * (1.0 / 110)))));
    } else {
        const double th = sqrt(th2);
        A = sin(th) / th;
        B = (1.0 - cos(th)) / th2;
        Cc = (th - sin(th)) / (th2 * th);
    }
    const double P[9] = {0, -p2, p1, p2, 0, -p0, -p1, p0, 0};
    double P2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += P[3 * i + k] * P[3 * k + j];
            P2[3 * i + j] = acc;
        }
    double R[9], V[9];
    for (int i = 0; i < 9; ++i) {
        const double I = (i % 4 == 0) ? 1.0 : 0.0;
        R[i] = I + A * P[i] + B * P2[i];
        V[i] = I + B * P[i] + Cc * P2[i];
    }
    double t[3];
    for (int i = 0; i < 3; ++i) t[i] = V[3 * i] * x[0] + V[3 * i + 1] * x[1] + V[3 * i + 2] * x[2];
    double out[16] = {0};
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 4; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * T[4 * k + j];
            out[4 * i + j] = acc + (j == 3 ? t[i] : 0.0);
        }
    }
    out[15] = 1.0;
    for (int i = 0; i < 16; ++i) T[i] = out[i];
}

// 1 / sqrt(d) for d > 0.  On the device: a float seed refined by two Newton
// steps y <- y (3 - d y^2) / 2 in FP64 (the relative error e becomes about
// 1.5 e^2 per step: 2e-7, 1e-13, then below double rounding), a short
// dependent chain where FP64 sqrt and division are long ones.
__host__ __device__ inline double inv_sqrt(double d)
{
#ifdef __CUDA_ARCH__
    if (d > 1e-30 && d < 1e30) {
        double y = (double)rsqrtf((float)d);
        y = y * (1.5 - 0.5 * d * y * y);
        y = y * (1.5 - 0.5 * d * y * y);
        return y;
    }
#endif
    return 1.0 / sqrt(d);
}

// Solve the symmetric positive definite 6x6 system A x = b (Cholesky, with
// the reciprocals of the diagonal of L); false when a pivot is not positive.
__host__ __device__ inline bool solve6(const double A[36], const double b[6], double x[6])
{
    double L[36] = {0}, inv[6];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            double acc = A[6 * i + j];
            for (int k = 0; k < j; ++k) acc -= L[6 * i + k] * L[6 * j + k];
            if (i == j) {
                if (!(acc > 0.0)) return false;
                inv[i] = inv_sqrt(acc);  // 1 / L_ii
            } else {
                L[6 * i + j] = acc * inv[j];
            }
        }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double acc = b[i];
        for (int k = 0; k < i; ++k) acc -= L[6 * i + k] * y[k];
        y[i] = acc * inv[i];
    }
    for (int i = 5; i >= 0; --i) {
        double acc = y[i];
        for (int k = i + 1; k < 6; ++k) acc -= L[6 * k + i] * x[k];
        x[i] = acc * inv[i];
    }
    return true;
}

}  // namespace mv
