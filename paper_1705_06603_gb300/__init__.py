"""GB300 (sm_103a) distributed shift-variant deblurring: the C-ABI library
``libdv`` and its thin Python binding (``paper_1705_06603_gb300.dv``).

Importing the package does not load the CUDA library; importing ``.dv`` does,
and fails loudly when the library has not been built."""
