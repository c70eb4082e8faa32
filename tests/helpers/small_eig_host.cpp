// Host build of the library's small dense eigensolver, for its CPU unit test.
#include <vector>

#include "small_eig.h"

extern "C" int small_eig_host(int m, double* A, double* w, double* V) {
  std::vector<bem::small::zc> Z((size_t)m * m);
  return bem::small::eig(m, reinterpret_cast<bem::small::zc*>(A),
                         reinterpret_cast<bem::small::zc*>(w),
                         reinterpret_cast<bem::small::zc*>(V), Z.data());
}
