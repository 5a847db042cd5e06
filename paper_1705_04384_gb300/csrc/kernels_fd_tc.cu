// Placeholder for the tensor-core FD path.
#include "context.h"

namespace iga {

struct TcFd {};

TcFd *make_tc_fd(int, int, int, const Factor1D &, cudaStream_t) {
  throw Error{IGA_ERR_UNSUPPORTED, "TF32/BF16 FD not built yet"};
}
void tc_fd_apply(TcFd &, IdxPtr<const double>, IdxPtr<float>, cudaStream_t) {
  throw Error{IGA_ERR_UNSUPPORTED, "TF32/BF16 FD not built yet"};
}
void tc_fd_apply_f64out(TcFd &, IdxPtr<const double>, double *, cudaStream_t) {
  throw Error{IGA_ERR_UNSUPPORTED, "TF32/BF16 FD not built yet"};
}
void destroy_tc_fd(TcFd *fd) { delete fd; }

}  // namespace iga
