// Serving runtime (continuous batching) -- filled in below.
#include "cd_internal.h"
