// Host-only export of the reference matrices for the build-time code generator
// (compiled with the host compiler into a helper library; not part of the runtime).
#include <cstdint>
#include <cstring>
#include <string>

#include "../tables.h"

extern "C" int yt_host_reference_matrix(int N, const char* name, double* out, int64_t* count) {
  try {
    const yt::RefMatrices& R = yt::reference_matrices(N);
    const std::string nm(name);
    const std::vector<double>* v = nullptr;
    if (nm == "Khat") v = &R.Khat;
    else if (nm == "Ktilde") v = &R.Ktilde;
    else if (nm == "R") v = &R.R;
    else if (nm == "Rhat") v = &R.Rhat;
    else if (nm == "f") v = &R.f;
    if (!v) return 1;
    *count = (int64_t)v->size();
    if (out) std::memcpy(out, v->data(), v->size() * sizeof(double));
    return 0;
  } catch (...) {
    return 2;
  }
}
