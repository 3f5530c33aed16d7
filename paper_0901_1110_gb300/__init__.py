"""GB300-native implicit radiation / ionization / gas-energy step (placeholder; binding follows)."""
