// Internal: event bracket around one kernel launch (active only while
// profiling is enabled through qdpg_profile_enable).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace qdpg {

class ProfScope {
 public:
  ProfScope(const char* name, cudaStream_t s);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  bool active_;
  size_t idx_;
  cudaStream_t s_;
};

}  // namespace qdpg
