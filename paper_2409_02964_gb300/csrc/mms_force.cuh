// mms_force.cuh -- GENERATED by gen_mms_force.py; do not edit by hand.
//
// Body force of Eq. (25) (constant density, pressure term dropped) for the
// spatiotemporal manufactured solution phi = phi0 + A sin(kx) sin(ky) cos(wt),
// phi u = grad psi + rot Psi (see the generator for the definitions), per unit rho0.
// Arguments: sx, cx = sin, cos of k x; sy, cy = sin, cos of k y; ct, st = cos, sin
// of w t. Evaluated from phi, q = phi u and their derivatives, u by the quotient rule.
// T is the arithmetic type (float or a packed pair); it must provide + - * between
// T values and with a float on either side, unary -, and mms_rcp(T).
#pragma once

namespace lbmv {

template <typename T>
__device__ __forceinline__ void mms_force(T sx, T cx, T sy, T cy, float ct, float st, float k, float w, float A,
                                          float U0, float phi0, float nu, T& fx, T& fy) {
    const float a = A * ct;
    const float b = -(A * w * st) / (2.0f * k);
    const float bt = -(A * w * w * ct) / (2.0f * k);
    const float ak = a * k;
    const float akk = a * k * k;
    const float bk = b * k;
    const float uk = U0 * k;
    const float kk = k * k;
    const T ss = sx * sy;
    const T cc = cx * cy;
    const T cs = cx * sy;
    const T sc = sx * cy;
    const T ph = phi0 + a * ss;
    const T phx = ak * cs;
    const T phy = ak * sc;
    const T phxx = -akk * ss;
    const T phxy = akk * cc;
    const T qx = b * cs + U0 * sc;
    const T qy = b * sc - U0 * cs;
    const T qxt = bt * cs;
    const T qyt = bt * sc;
    const T qxx = uk * cc - bk * ss;
    const T qxy = bk * cc - uk * ss;
    const T qyx = bk * cc + uk * ss;
    const T qyy = -bk * ss - uk * cc;
    const T qmx = -kk * (b * sc + U0 * cs);
    const T qmy = kk * (U0 * sc - b * cs);
    const T ip = mms_rcp(ph);
    const T ux = qx * ip;
    const T uy = qy * ip;
    const T uxx = (qxx - ux * phx) * ip;
    const T uxy = (qxy - ux * phy) * ip;
    const T uyx = (qyx - uy * phx) * ip;
    const T uyy = (qyy - uy * phy) * ip;
    const T uxXX = (-kk * qx - 2.0f * uxx * phx - ux * phxx) * ip;
    const T uxYY = (-kk * qx - 2.0f * uxy * phy - ux * phxx) * ip;
    const T uxXY = (qmx - uxx * phy - uxy * phx - ux * phxy) * ip;
    const T uyXX = (-kk * qy - 2.0f * uyx * phx - uy * phxx) * ip;
    const T uyYY = (-kk * qy - 2.0f * uyy * phy - uy * phxx) * ip;
    const T uyXY = (qmy - uyx * phy - uyy * phx - uy * phxy) * ip;
    const T dv = uxx + uyy;
    const T txx = 2.0f * uxx - (2.0f / 3.0f) * dv;
    const T tyy = 2.0f * uyy - (2.0f / 3.0f) * dv;
    const T txy = uxy + uyx;
    const T dxtxx = (4.0f / 3.0f) * uxXX - (2.0f / 3.0f) * uyXY;
    const T dytyy = (4.0f / 3.0f) * uyYY - (2.0f / 3.0f) * uxXY;
    const T dytxy = uxYY + uyXY;
    const T dxtxy = uxXY + uyXX;
    const T vx = phx * txx + ph * dxtxx + phy * txy + ph * dytxy;
    const T vy = phx * txy + ph * dxtxy + phy * tyy + ph * dytyy;
    fx = qxt + qxx * ux + qx * uxx + qxy * uy + qx * uyy - nu * vx;
    fy = qyt + qyx * ux + qy * uxx + qyy * uy + qy * uyy - nu * vy;
}

}  // namespace lbmv
