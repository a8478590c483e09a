// FP64 instantiations of the subvolume kernels.
#include "k_subvol.cuh"
namespace la {
template <>
cudaError_t launch_factor<double>(const LevelGeom& L, const FineOp* fine, const double* sigma, const TimeMats* tm,
                                  double2* factors, int* status, cudaStream_t s) {
#define LA_CALL(N) launch_factor_n<double, N>(L, fine, sigma, tm, factors, status, s)
  {
#define LA_WCALL(N) launch_factor_wide_n<double, N>(L, fine, tm, factors, status, s)
    LA_NPAD_DISPATCH_WIDE(L.npad, LA_WCALL)
#undef LA_WCALL
  }
  LA_NPAD_DISPATCH(L.npad, LA_CALL)
#undef LA_CALL
}
template <>
cudaError_t launch_sweep_fine<double>(const LevelGeom& L, const FineOp& g, const TimeMats* tm, int K, const double2* f,
                                      const double2* yx, double2* c, const double2* factors, int colour, int* status, cudaStream_t s) {
#define LA_CALL(N) launch_sweep_fine_n<double, N>(L, g, tm, K, f, yx, c, factors, colour, status, s)
  LA_NPAD_DISPATCH_WIDE(L.npad, LA_CALL)
  LA_NPAD_DISPATCH(L.npad, LA_CALL)
#undef LA_CALL
}
template <>
cudaError_t launch_sweep_coarse<double>(const LevelGeom& L, const double* sigma, const TimeMats* tm, int K,
                                        const double2* gvec, double2* e, const double2* factors, int colour,
                                        int* status, cudaStream_t s) {
#define LA_CALL(N) launch_sweep_coarse_n<double, N>(L, sigma, tm, K, gvec, e, factors, colour, status, s)
  LA_NPAD_DISPATCH(L.npad, LA_CALL)
#undef LA_CALL
}
template <>
cudaError_t launch_gresid_tiles<double>(const LevelGeom& L, const double* sigma, const TimeMats* tm, int K,
                                     const double2* gvec, const double2* e, double2* out, cudaStream_t s) {
  return launch_gresid_tiles_r<double>(L, sigma, tm, K, gvec, e, out, s);
}
}  // namespace la
