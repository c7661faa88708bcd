// drt_k_batch_redo_dual.cu -- the batch redo kernel with rates (Doppler output), its own translation unit
#define DRT_BATCH_REDO_DUAL
#include "drt_k_batch_redo.cu"
