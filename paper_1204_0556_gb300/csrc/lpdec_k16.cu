#define LPDEC_D 16
#include "lpdec_kclass.cuh"
