// FP32 (complex64) instantiations of the subvolume kernels.
#include "k_subvol.cuh"
namespace la {
template <>
cudaError_t launch_factor<float>(const LevelGeom& L, const FineOp* fine, const float* sigma, const TimeMats* tm,
                                  float2* factors, int* status, cudaStream_t s) {
#define LA_CALL(N) launch_factor_blk_n<float, N>(L, fine, sigma, tm, factors, status, s)
  {
#define LA_WCALL(N) launch_factor_wide_n<float, N>(L, fine, tm, factors, status, s)
    LA_NPAD_DISPATCH_WIDE(L.npad, LA_WCALL)
#undef LA_WCALL
  }
  LA_NPAD_DISPATCH(L.npad, LA_CALL)
#undef LA_CALL
}
template <>
cudaError_t launch_sweep_fine<float>(const LevelGeom& L, const FineOp& g, const TimeMats* tm, int K, const float2* f,
                                      const float2* yx, float2* c, const float2* factors, int colour, int* status, cudaStream_t s) {
#define LA_CALL(N) launch_sweep_fine_n<float, N>(L, g, tm, K, f, yx, c, factors, colour, status, s)
  LA_NPAD_DISPATCH_WIDE(L.npad, LA_CALL)
  LA_NPAD_DISPATCH(L.npad, LA_CALL)
#undef LA_CALL
}
template <>
cudaError_t launch_sweep_coarse<float>(const LevelGeom& L, const float* sigma, const TimeMats* tm, int K,
                                        const float2* gvec, float2* e, const float2* factors, int colour,
                                        int* status, cudaStream_t s) {
#define LA_CALL(N) launch_sweep_coarse_n<float, N>(L, sigma, tm, K, gvec, e, factors, colour, status, s)
  LA_NPAD_DISPATCH(L.npad, LA_CALL)
#undef LA_CALL
}
template <>
cudaError_t launch_gresid_tiles<float>(const LevelGeom& L, const float* sigma, const TimeMats* tm, int K,
                                     const float2* gvec, const float2* e, float2* out, cudaStream_t s) {
  return launch_gresid_tiles_r<float>(L, sigma, tm, K, gvec, e, out, s);
}
}  // namespace la
