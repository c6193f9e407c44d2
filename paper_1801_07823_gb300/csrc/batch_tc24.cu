// Instantiations of the tensor-core batched coarsest CGNE for nc = 24.
#include "batch_tc.cuh"

bool swtc::run_nc24(const TcArgs& a, int K, int S, bool f32, int device, cudaStream_t s,
                     int sms_use) {
  return run_nc<24>(a, K, S, f32, device, s, sms_use);
}
