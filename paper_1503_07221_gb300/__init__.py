"""GB300 (sm_103a) assembler of the space-time Galerkin system of the
time-domain hypersingular operator: C-ABI library libtdbem plus a thin
ctypes binding (tdbem) and seeded synthetic inputs (inputs)."""
