// The outer-block panel kernel for FP32 fronts, in a translation unit of its
// own so that the two front types compile in parallel.
#include "block_panels.cuh"

namespace sgn {

template void launch_block_panels<float, 16>(unsigned, size_t, cudaStream_t, const DevSym &, const SV &,
                                          const int32_t *, const BandItem *, int, int, double,
                                          unsigned long long *, unsigned *, int *);
template void launch_block_panels<float, 32>(unsigned, size_t, cudaStream_t, const DevSym &, const SV &,
                                          const int32_t *, const BandItem *, int, int, double,
                                          unsigned long long *, unsigned *, int *);
template void set_block_panels_smem<float, 16>(int);
template void set_block_panels_smem<float, 32>(int);

}  // namespace sgn
