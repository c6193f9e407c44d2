// Instantiations of the tensor-core batched coarsest CGNE for nc = 16.
#include "batch_tc.cuh"

bool swtc::run_nc16(const TcArgs& a, int K, int S, bool f32, int device, cudaStream_t s,
                     int sms_use) {
  return run_nc<16>(a, K, S, f32, device, s, sms_use);
}
