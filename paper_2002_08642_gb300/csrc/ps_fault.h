// ps_fault.h -- host-side fault injection for the library's error paths.
// PS_FAULT_ALLOC=ctx (ps_init), ms (ps_ms_create) or all makes the named
// host allocation fail as if the allocator returned nothing, so that the
// PS_ENOMEM paths can be exercised by tests without any GPU fault.
#ifndef PS_FAULT_H
#define PS_FAULT_H

#include <stdlib.h>
#include <string.h>

static inline bool ps_fault_alloc(const char* what) {
    const char* e = getenv("PS_FAULT_ALLOC");
    return e && (!strcmp(e, "all") || !strcmp(e, what));
}

#endif
