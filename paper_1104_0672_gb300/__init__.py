"""ARKCoS ring-band sphere convolution for GB300 (placeholder, binding added below)."""
