"""User integrand sources shared by the user-integrand tests."""
COSPROD = r'''
__device__ float zmc_user_g32(const float* y, const float* x) {
  float g = 1.0f;
  for (int k = 0; k < ZMC_N; ++k) g *= __cosf(x[k] * y[k]);
  return g;
}
__device__ double zmc_user_g64(const double* y, const double* x) {
  double g = 1.0;
  for (int k = 0; k < ZMC_N; ++k) g *= cos(x[k] * y[k]);
  return g;
}
'''

# g = (sum_l x_l) * prod_k y_k: on [0, b_1] x ... the integral is
# (sum x) * prod_k b_k^2 / 2.
SUMX_PRODY = r'''
__device__ float zmc_user_g32(const float* y, const float* x) {
  float s = 0.0f, p = 1.0f;
  for (int l = 0; l < ZMC_M; ++l) s += x[l];
  for (int k = 0; k < ZMC_N; ++k) p *= y[k];
  return s * p;
}
'''

BROKEN = "__device__ float zmc_user_g32(const float* y, const float* x) { return y[0] +; }"
