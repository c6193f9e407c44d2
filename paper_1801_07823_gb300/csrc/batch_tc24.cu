// Instantiations of the tensor-core batched coarsest CGNE for nc = 24.
#include "batch_tc.cuh"

bool swtc::run_nc24(const TcArgs& a, int K, int S, int device, cudaStream_t s) {
  return run_nc<24>(a, K, S, device, s);
}
