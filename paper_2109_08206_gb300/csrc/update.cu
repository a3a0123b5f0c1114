// Configuration update after the solve (Appendix Eq. constrainedeom_euler a-c):
//   U = M (F_nc + D gamma) = U_nc + U_c,   C^{k+1} = C^k + h G U,
// with G = diag(I_3, Psi(theta)) and Psi(theta) Omega = 1/2 [-v.Omega ; s Omega - v x Omega]
// for theta = (s, v) (the paper's P_ij = eps_ikj p_k gives P Omega = v x Omega).
// The centre is wrapped back into [0, box) and the quaternion renormalised.
// One thread per rod; x and quat are updated in place.
#include "internal.cuh"

namespace alens {

template <typename T>
__global__ void k_update(int n, int np, bool have_uc, Geo g0, const SysGeo* __restrict__ systab,
                         const int* __restrict__ sysid, const int* __restrict__ flags,
                         const double* __restrict__ xw, const double* __restrict__ unc, const T* __restrict__ Uref,
                         const T* __restrict__ dU, const int* __restrict__ rank, double* __restrict__ x,
                         double* __restrict__ quat, double* __restrict__ vel_out,
                         const unsigned long long* __restrict__ mdev)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flags[F_ERR] != 0 || flags[F_SOLVE_ERR] != 0) return;   // leave the state untouched after a failure
    if (mdev) have_uc = *mdev > 0;   // a step without readbacks: the device's constraint count
    const Geo& g = geo_of(g0, systab, sysid, i);
    double U[6];
    const int r = rank ? rank[i] : i;   // the solver's position of rod i
#pragma unroll
    for (int u = 0; u < 6; ++u) {
        U[u] = unc[u * (size_t)np + i];
        if (have_uc) {
            // M D gamma = Uref + M D delta (every reference pass clears the increment)
            U[u] += (double)Uref[6 * (size_t)r + u] + (double)dU[6 * (size_t)r + u];
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) x[3 * (size_t)i + k] = wrap_coord(xw[k * (size_t)np + i] + g.dt * U[k], g.box[k]);
    double s = quat[4 * (size_t)i], v0 = quat[4 * (size_t)i + 1], v1 = quat[4 * (size_t)i + 2],
           v2 = quat[4 * (size_t)i + 3];
    double o0 = U[3], o1 = U[4], o2 = U[5];
    double vxo0 = v1 * o2 - v2 * o1, vxo1 = v2 * o0 - v0 * o2, vxo2 = v0 * o1 - v1 * o0;
    double hh = 0.5 * g.dt;
    double n0 = s - hh * (v0 * o0 + v1 * o1 + v2 * o2);
    double n1 = v0 + hh * (s * o0 - vxo0);
    double n2 = v1 + hh * (s * o1 - vxo1);
    double n3 = v2 + hh * (s * o2 - vxo2);
    double inv = 1.0 / sqrt(n0 * n0 + n1 * n1 + n2 * n2 + n3 * n3);
    quat[4 * (size_t)i] = n0 * inv;
    quat[4 * (size_t)i + 1] = n1 * inv;
    quat[4 * (size_t)i + 2] = n2 * inv;
    quat[4 * (size_t)i + 3] = n3 * inv;
    if (vel_out) {
#pragma unroll
        for (int u = 0; u < 6; ++u) vel_out[6 * (size_t)i + u] = U[u];
    }
}

cudaError_t launch_update(aLENS_ctx* ctx, int n, int m, double* x, double* quat, int precision, double* vel_out,
                          const int* rank)
{
    if (n <= 0) return cudaSuccess;
    int b = (n + 255) / 256;
    int np = (int)ctx->max_rods;
    if (precision == ALENS_MIXED) {
        k_update<float><<<b, 256, 0, ctx->stream>>>(n, np, m > 0, ctx->geo, ctx->cur_systab, ctx->cur_sysid, ctx->dflags, ctx->xw, ctx->unc, ctx->sb32.Uref, ctx->sb32.U, rank, x, quat,
                                                    vel_out, ctx->mdev);
        ++ctx->launches;
    } else {
        k_update<double><<<b, 256, 0, ctx->stream>>>(n, np, m > 0, ctx->geo, ctx->cur_systab, ctx->cur_sysid, ctx->dflags, ctx->xw, ctx->unc, ctx->sb64.Uref, ctx->sb64.U, rank, x, quat,
                                                     vel_out, ctx->mdev);
        ++ctx->launches;
    }
    return cudaGetLastError();
}

}  // namespace alens
