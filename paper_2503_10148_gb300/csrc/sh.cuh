// Real spherical harmonics up to degree 3 as polynomials of a unit direction
// (x, y, z), index l*l + l + m, Condon-Shortley phase included.
//
// Each Y_{l,m} = K_l^|m| P_l^|m|(z) {cos, sin}(|m| phi) (times sqrt 2 for
// m != 0), with P_l^m(z) = Q_l^m(z) (1 - z^2)^{m/2} and
// (1 - z^2)^{m/2} e^{i m phi} = (x + i y)^m on the unit sphere; expanding the
// Legendre polynomials Q for l <= 3 gives the forms below.  The constants are
// the normalisations sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) times sqrt 2 (m != 0)
// times the leading coefficient of Q.  sh_grad returns the gradient of these
// polynomials in R^3; callers project it onto the sphere.
#pragma once

namespace sss {

constexpr float kY00 = 0.28209479177387814f;  // 1 / (2 sqrt(pi))
constexpr float kY1 = 0.4886025119029199f;    // sqrt(3 / (4 pi))
constexpr float kY2a = 1.0925484305920792f;   // sqrt(15 / (4 pi))
constexpr float kY2b = 0.31539156525252005f;  // sqrt(5 / (16 pi))
constexpr float kY2c = 0.5462742152960396f;   // sqrt(15 / (16 pi))
constexpr float kY3a = 0.5900435899266435f;   // sqrt(35 / (32 pi))
constexpr float kY3b = 2.890611442640554f;    // sqrt(105 / (4 pi))
constexpr float kY3c = 0.4570457994644658f;   // sqrt(21 / (32 pi))
constexpr float kY3d = 0.3731763325901154f;   // sqrt(7 / (16 pi))
constexpr float kY3e = 1.445305721320277f;    // sqrt(105 / (16 pi))

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
  Y[0] = kY00;
  if (DEG >= 1) {
    Y[1] = -kY1 * y;
    Y[2] = kY1 * z;
    Y[3] = -kY1 * x;
  }
  if (DEG >= 2) {
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kY2a * x * y;
    Y[5] = -kY2a * y * z;
    Y[6] = kY2b * (3.0f * zz - 1.0f);
    Y[7] = -kY2a * x * z;
    Y[8] = kY2c * (xx - yy);
    if (DEG >= 3) {
      Y[9] = -kY3a * y * (3.0f * xx - yy);
      Y[10] = kY3b * x * y * z;
      Y[11] = -kY3c * y * (5.0f * zz - 1.0f);
      Y[12] = kY3d * z * (5.0f * zz - 3.0f);
      Y[13] = -kY3c * x * (5.0f * zz - 1.0f);
      Y[14] = kY3e * z * (xx - yy);
      Y[15] = -kY3a * x * (xx - 3.0f * yy);
    }
  }
}

// d/d(x,y,z) of sum_k w[k] Y_k(x, y, z).
template <int DEG>
__device__ __forceinline__ void sh_grad(float x, float y, float z, const float* w, float& gx, float& gy,
                                        float& gz) {
  gx = gy = gz = 0.0f;
  if (DEG >= 1) {
    gy -= kY1 * w[1];
    gz += kY1 * w[2];
    gx -= kY1 * w[3];
  }
  if (DEG >= 2) {
    gx += kY2a * y * w[4];
    gy += kY2a * x * w[4];
    gy -= kY2a * z * w[5];
    gz -= kY2a * y * w[5];
    gz += 6.0f * kY2b * z * w[6];
    gx -= kY2a * z * w[7];
    gz -= kY2a * x * w[7];
    gx += 2.0f * kY2c * x * w[8];
    gy -= 2.0f * kY2c * y * w[8];
    if (DEG >= 3) {
      float xx = x * x, yy = y * y, zz = z * z;
      gx -= 6.0f * kY3a * x * y * w[9];
      gy -= 3.0f * kY3a * (xx - yy) * w[9];
      gx += kY3b * y * z * w[10];
      gy += kY3b * x * z * w[10];
      gz += kY3b * x * y * w[10];
      gy -= kY3c * (5.0f * zz - 1.0f) * w[11];
      gz -= 10.0f * kY3c * y * z * w[11];
      gz += kY3d * (15.0f * zz - 3.0f) * w[12];
      gx -= kY3c * (5.0f * zz - 1.0f) * w[13];
      gz -= 10.0f * kY3c * x * z * w[13];
      gx += 2.0f * kY3e * x * z * w[14];
      gy -= 2.0f * kY3e * y * z * w[14];
      gz += kY3e * (xx - yy) * w[14];
      gx -= 3.0f * kY3a * (xx - yy) * w[15];
      gy += 6.0f * kY3a * x * y * w[15];
    }
  }
}

}  // namespace sss
