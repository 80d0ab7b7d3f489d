// tcgen05 tensor-core contraction (placeholder until the kernel lands).
#include <cuda_runtime.h>
#include "coffee_internal.h"
namespace coffee {
int tc_supported(int, int, int, int) { return 0; }
void build_tc_image(int, int, int, int, std::vector<uint8_t>& img, TcTable& meta) { img.clear(); meta = TcTable{}; }
int launch_tc(int, int, const TcParams&, int, void*, std::string& why) { why = "not built"; return (int)cudaErrorNotSupported; }
}
