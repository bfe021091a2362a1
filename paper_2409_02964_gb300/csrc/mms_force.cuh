// mms_force.cuh -- GENERATED by gen_mms_force.py; do not edit by hand.
//
// Body force of Eq. (25) (constant density, pressure term dropped) for the
// spatiotemporal manufactured solution phi = phi0 + A sin(kx) sin(ky) cos(wt),
// phi u = grad psi + rot Psi (see the generator for the definitions). Arguments:
// sx, cx = sin, cos of k x; sy, cy = sin, cos of k y; ct, st = cos, sin of w t.
// T is the arithmetic type (float or a packed pair); it must provide + and *
// between T values and with a float on either side, and mms_rcp(T).
#pragma once

namespace lbmv {

template <typename T>
__device__ __forceinline__ void mms_force(T sx, T cx, T sy, T cy, float ct, float st, float k, float w, float A,
                                          float U0, float phi0, float nu, T& fx, T& fy) {
    const T e0 = (cx * sy);
    const T e1 = (A * e0);
    const T e2 = (ct * e1);
    const T e3 = (A * sx);
    const T e4 = (ct * e3);
    const T e5 = (e4 * sy);
    const T e6 = (e5 + phi0);
    const T e7 = (e6 * e6);
    const T e8 = ((w * w) * e7);
    const float e9 = (2.0f * U0 * k);
    const T e10 = (e9 * sx);
    const T e11 = (cy * e10);
    const float e12 = (st * w);
    const T e13 = (e12 * e1);
    const T e14 = (e13 + (-1.0f * e11));
    const T e15 = (e9 * e0);
    const T e16 = (e12 * cy);
    const T e17 = (e16 * e3);
    const T e18 = (e15 + e17);
    const T e19 = (3.0f * e18);
    const T e20 = (cy * e4);
    const T e21 = (A * cx * e16);
    const T e22 = (e21 + (e10 * sy));
    const T e23 = (e9 * cx * cy);
    const T e24 = (e12 * e3 * sy);
    const T e25 = (e24 + (-1.0f * e23));
    const T e26 = (e25 * e6);
    const T e27 = (3.0f * e14);
    const T e28 = (e6 * (e23 + e24));
    const T e29 = (6.0f * e14);
    const float e30 = ((ct * ct) * (A * A));
    const T e31 = (2.0f * e30 * cy * e0 * sx);
    const T e32 = (e21 + (-2.0f * U0 * k * sx * sy));
    const T e33 = (7.0f * e5);
    const float e34 = (8.0f * e30);
    const T e35 = ((cx * cx) * (sy * sy));
    const T e36 = ((cy * cy) * (sx * sx));
    const T e37 = (-1.0f * e14);
    const T e38 = (2.0f * e2);
    const T e39 = ((-3.0f * e18 * e2) + (3.0f * e22 * e6) + (3.0f * e32 * e6) + (3.0f * ct * A * cy * e37 * sx));
    const float e40 = (2.0f * nu * (k * k));
    const T e41 = ((0.08333333333333333f) * mms_rcp(e7 * k));
    const T e42 = (e14 * e2);
    const T e43 = (6.0f * e18);
    fx = (-1.0f * e41 * ((e26 * e27) + (e28 * e29) + (e40 * ((e7 * (e11 + e13)) + (-1.0f * e18 * e31) + (-1.0f * e2 * e26) + (-1.0f * e20 * e39) + (-1.0f * e38 * (e26 + (-2.0f * e28) + (e18 * e20) + (e37 * e38))) + (-8.0f * e2 * e28) + (7.0f * e14 * e7) + (-1.0f * e14 * e33 * e6) + (-1.0f * e34 * e14 * e35) + (-1.0f * e30 * e29 * e36) + (ct * A * cx * cy * e18 * e6) + (ct * A * cy * e32 * e6 * sx) + (6.0f * ct * A * cy * e22 * e6 * sx))) + (3.0f * e2 * (e14 * e14)) + (6.0f * e2 * e8) + (e14 * e19 * e20) + (-1.0f * e19 * e22 * e6)));
    fy = (-1.0f * e41 * ((e19 * e28) + (e19 * e42) + (e26 * e43) + (e40 * ((e7 * (e17 + (-1.0f * e15))) + (-1.0f * e14 * e31) + (-1.0f * e2 * e39) + (-1.0f * e20 * e28) + (-8.0f * e20 * e26) + (7.0f * e18 * e7) + (-1.0f * e18 * e33 * e6) + (-1.0f * e34 * e18 * e36) + (-1.0f * e30 * e35 * e43) + (2.0f * ct * A * cy * sx * ((-1.0f * e28) + (-1.0f * e42) + (2.0f * e25 * e6) + (2.0f * ct * A * cy * e18 * sx))) + (ct * A * cx * cy * e14 * e6) + (ct * A * cx * e22 * e6 * sy) + (6.0f * ct * A * cx * e32 * e6 * sy))) + (3.0f * e20 * (e18 * e18)) + (6.0f * e20 * e8) + (-1.0f * e27 * e32 * e6)));
}

}  // namespace lbmv
