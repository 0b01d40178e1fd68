// The emulation's globals for the library built whole for the host (the
// harness binaries define their own), and a counter the tests read.
#include "shim.h"
thread_local dim threadIdx, blockIdx;
dim blockDim, gridDim;
thread_local WarpCtx *tw;

// CUDA graphs launched so far (each replay of a captured launch sequence)
extern "C" long long emu_graph_launch_count() { return emu_graph_launches; }
