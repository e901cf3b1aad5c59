// FP32 Tensor-Memory row / entropy-epilogue kernel over several units (rotation
// angles) for transform sizes 512, 1024 and 2048.
#include "pipeline_impl.cuh"
namespace cmif {
template <int Q, bool NMI>
cudaError_t launch_rows_tm_units(const Geom& g, const PipeArgs<float>& a, cudaStream_t s) {
    auto kern = k_pair_rows_tm<Q, NMI, 1>;
    cudaError_t e = ensure_smem(kern, RowTmCfg<Q>::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<a.rows_grid, RowTmCfg<Q>::THREADS, RowTmCfg<Q>::SMEM, s>>>(a.Y, g, a.tw, a.mi, a.n, a.st, a.tm_cols,
                                                                     kDefaultWaitPolls, -1, 0, nullptr, nullptr,
                                                                     nullptr);
    return cudaGetLastError();
}
template cudaError_t launch_rows_tm_units<512, false>(const Geom&, const PipeArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_tm_units<512, true>(const Geom&, const PipeArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_tm_units<1024, false>(const Geom&, const PipeArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_tm_units<1024, true>(const Geom&, const PipeArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_tm_units<2048, false>(const Geom&, const PipeArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_tm_units<2048, true>(const Geom&, const PipeArgs<float>&, cudaStream_t);
}  // namespace cmif
