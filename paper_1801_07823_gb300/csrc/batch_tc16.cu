// Instantiations of the tensor-core batched coarsest CGNE for nc = 16.
#include "batch_tc.cuh"

bool swtc::run_nc16(const TcArgs& a, int K, int S, int device, cudaStream_t s) {
  return run_nc<16>(a, K, S, device, s);
}
